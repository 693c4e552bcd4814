// Device building blocks of the finite-volume step: primitive recovery (Eq. 2), the MC-limited
// MUSCL face states (App. A.1) and the HLLC flux with Davis wave speeds (App. A.2).
// Templated on the working precision `real` (float for production, double for parity runs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dh {

// Status bits of the device step record.
enum : unsigned {
  FLAG_NONFINITE = 1u,
  FLAG_POSITIVITY = 2u,
  FLAG_MG_NOCONV = 4u,
  FLAG_COOL_CAP = 8u,   // informational: a cell hit the substep cap
};
constexpr unsigned FATAL_FLAGS = FLAG_NONFINITE | FLAG_POSITIVITY | FLAG_MG_NOCONV;

// Device-resident record of the time integration (one per context).
struct StepRecord {
  double dt;             // dt of the step in flight / last step
  double t;              // simulation time after the last step
  long long nstep;       // completed steps
  unsigned flags;        // FLAG_* bits
  int fail_step;         // step index of the first fatal failure, -1 if none
  unsigned long long cfl_min_bits;  // min over cells of dx_a/(|v_a|+c) as ordered bits
  double ou_norm;        // a_rms / sqrt(<|a|^2>) of the current forcing table
};

__host__ __device__ inline int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename real> struct Prim { real r, vx, vy, vz, p; };

// Quotients and square roots of the working precision.  The float64 instance (parity runs)
// keeps IEEE division and square root; the float32 production instance uses the hardware
// approximations (reciprocal and reciprocal square root, a few ulp), whose error stays far
// below the float32 parity tolerance.  Host builds always use the IEEE operations.
__host__ __device__ __forceinline__ double q_div(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ double q_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float q_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
__host__ __device__ __forceinline__ float q_sqrt(float x) {
#ifdef __CUDA_ARCH__
  return x * rsqrtf(x);
#else
  return sqrtf(x);
#endif
}

// W = (rho, v, P) from U (Eq. 2).
template <typename real>
__host__ __device__ __forceinline__ Prim<real> cons_to_prim(real r, real mx, real my, real mz, real E,
                                                   real gm1) {
  Prim<real> w;
  w.r = r;
  w.vx = q_div(mx, r);
  w.vy = q_div(my, r);
  w.vz = q_div(mz, r);
  w.p = gm1 * (E - real(0.5) * r * (w.vx * w.vx + w.vy * w.vy + w.vz * w.vz));
  return w;
}

// MC(a, b) = 0 if a*b <= 0 else sign(a) min(2|a|, 2|b|, |a+b|/2)  (App. A.1, MC limiter).
template <typename real>
__host__ __device__ __forceinline__ real mc_slope(real a, real b) {
  real m = fmin(fmin(real(2) * fabs(a), real(2) * fabs(b)), real(0.5) * fabs(a + b));
  return (a * b > real(0)) ? copysign(m, a) : real(0);
}

// Limited slope of a cell from its two neighbours along one axis, with the positivity fallback:
// if W +- dW/2 has rho <= 0 or P <= 0 every slope of the cell on that axis is zero.
template <typename real>
__host__ __device__ __forceinline__ Prim<real> limited_slope(const Prim<real>& wm, const Prim<real>& w0,
                                                    const Prim<real>& wp) {
  Prim<real> d;
  d.r = mc_slope(wp.r - w0.r, w0.r - wm.r);
  d.vx = mc_slope(wp.vx - w0.vx, w0.vx - wm.vx);
  d.vy = mc_slope(wp.vy - w0.vy, w0.vy - wm.vy);
  d.vz = mc_slope(wp.vz - w0.vz, w0.vz - wm.vz);
  d.p = mc_slope(wp.p - w0.p, w0.p - wm.p);
  const real hr = real(0.5) * d.r, hp = real(0.5) * d.p;
  const bool bad = (w0.r + hr <= real(0)) || (w0.p + hp <= real(0)) || (w0.r - hr <= real(0)) ||
                   (w0.p - hp <= real(0));
  if (bad) d = Prim<real>{real(0), real(0), real(0), real(0), real(0)};
  return d;
}

template <typename real>
__host__ __device__ __forceinline__ Prim<real> add_half(const Prim<real>& w, const Prim<real>& d, real s) {
  // w + s * d / 2 with s = +1 (left state of the upper face) or -1 (right state of the lower face)
  const real h = real(0.5) * s;
  return Prim<real>{w.r + h * d.r, w.vx + h * d.vx, w.vy + h * d.vy, w.vz + h * d.vz,
                    w.p + h * d.p};
}

// Flux components in the face frame: (mass, normal momentum, tangential 1, tangential 2, energy).
template <typename real> struct Flux { real f0, fn, ft1, ft2, fe; };

// HLLC flux (Toro, Spruce & Speares 1994) for face-frame states (rho, u_n, u_t1, u_t2, P).
// Region choice: S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; otherwise F_R.
template <typename real>
__host__ __device__ __forceinline__ Flux<real> hllc(real rL, real uL, real aL, real bL, real pL, real rR,
                                           real uR, real aR, real bR, real pR, real gamma,
                                           real gm1) {
  const real cL = q_sqrt(q_div(gamma * pL, rL));
  const real cR = q_sqrt(q_div(gamma * pR, rR));
  const real SL = fmin(uL - cL, uR - cR);
  const real SR = fmax(uL + cL, uR + cR);
  const real dL = SL - uL, dR = SR - uR;
  const real Sstar = q_div(pR - pL + rL * uL * dL - rR * uR * dR, rL * dL - rR * dR);

  // Select the side K whose (star) flux is taken.
  const bool left = (SL >= real(0)) || (Sstar >= real(0));
  const bool star = !(SL >= real(0)) && (Sstar >= real(0) || SR > real(0));
  const real r = left ? rL : rR, u = left ? uL : uR, a = left ? aL : aR, b = left ? bL : bR;
  const real p = left ? pL : pR, S = left ? SL : SR, d = left ? dL : dR;

  const real E = q_div(p, gm1) + real(0.5) * r * (u * u + a * a + b * b);
  const real mass = r * u;
  Flux<real> F{mass, mass * u + p, mass * a, mass * b, u * (E + p)};
  if (star) {
    const real coef = q_div(r * d, S - Sstar);
    const real Es = coef * (q_div(E, r) + (Sstar - u) * (Sstar + q_div(p, r * d)));
    F.f0 += S * (coef - r);
    F.fn += S * (coef * Sstar - mass);
    F.ft1 += S * (coef * a - r * a);
    F.ft2 += S * (coef * b - r * b);
    F.fe += S * (Es - E);
  }
  return F;
}

// HLLC flux across a face normal to `axis` (0 = x, 1 = y, 2 = z) from reconstructed
// primitive states; returns fluxes in (rho, m_x, m_y, m_z, E) order.
template <typename real>
__host__ __device__ __forceinline__ void face_flux(int axis, const Prim<real>& L, const Prim<real>& R,
                                          real gamma, real gm1, real out[5]) {
  if (axis == 0) {
    Flux<real> F = hllc(L.r, L.vx, L.vy, L.vz, L.p, R.r, R.vx, R.vy, R.vz, R.p, gamma, gm1);
    out[0] = F.f0; out[1] = F.fn; out[2] = F.ft1; out[3] = F.ft2; out[4] = F.fe;
  } else if (axis == 1) {
    Flux<real> F = hllc(L.r, L.vy, L.vx, L.vz, L.p, R.r, R.vy, R.vx, R.vz, R.p, gamma, gm1);
    out[0] = F.f0; out[1] = F.ft1; out[2] = F.fn; out[3] = F.ft2; out[4] = F.fe;
  } else {
    Flux<real> F = hllc(L.r, L.vz, L.vx, L.vy, L.p, R.r, R.vz, R.vx, R.vy, R.p, gamma, gm1);
    out[0] = F.f0; out[1] = F.ft1; out[2] = F.ft2; out[3] = F.fn; out[4] = F.fe;
  }
}

// Positive floating-point values order like their bit patterns as unsigned integers.
__device__ __forceinline__ unsigned long long ordered_bits(float x) {
  return (unsigned long long)__float_as_uint(x);
}
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

}  // namespace dh
