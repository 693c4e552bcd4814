// Device building blocks of the finite-volume step: primitive recovery (Eq. 2), the MC-limited
// MUSCL face states (App. A.1) and the HLLC flux with Davis wave speeds (App. A.2).
// Templated on the working precision `real` (float for production, double for parity runs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dh {

// Status bits of the device step record.
enum : unsigned {
  FLAG_NONFINITE = 1u,
  FLAG_POSITIVITY = 2u,
  FLAG_MG_NOCONV = 4u,
  FLAG_COOL_CAP = 8u,   // informational: a cell hit the substep cap
  FLAG_TIMEOUT = 16u,   // a bounded wait on the kernel's own copies gave up
};
constexpr unsigned FATAL_FLAGS = FLAG_NONFINITE | FLAG_POSITIVITY | FLAG_MG_NOCONV | FLAG_TIMEOUT;

// Device-resident record of the time integration (one per context).
struct StepRecord {
  double dt;             // dt of the step in flight / last step
  double t;              // simulation time after the last step
  long long nstep;       // completed steps
  unsigned flags;        // FLAG_* bits
  int fail_step;         // step index of the first fatal failure, -1 if none
  unsigned long long cfl_min_bits;  // min over cells of dx_a/(|v_a|+c) as ordered bits
  double ou_norm;        // a_rms / sqrt(<|a|^2>) of the current forcing table
  int cool_nsub_max;     // largest cooling substep count (> 1) since the last metrics read
  unsigned long long slope_fallbacks;  // positivity fallbacks (cell, axis, stage) since the last read
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

// ---- packed float32 pairs (FADD2 / FMUL2 / FFMA2 of sm_100+) ---------------------------------
// Each lane is an IEEE round-to-nearest float32 operation, so a packed expression gives the
// bits of the same scalar expression; packing halves the instruction count of paired work
// (the two sides of a face, two state components).  Float32 device code only.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b in one packed instruction: fma(b, -1, a) rounds the exact difference once.
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }

// Scalar products, sums and fused multiply-adds with their rounding spelled out.  The compiler
// never contracts these into other operations, so every inlined copy of a formula rounds the
// same way wherever it is called (a cell's flux does not depend on which loop phase of the
// stencil evaluates it).
__host__ __device__ __forceinline__ float rmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float radd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float rfma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
__host__ __device__ __forceinline__ double rmul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ double radd(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ double rfma(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return fma(a, b, c);
#endif
}

// W = (rho, v, P) from U (Eq. 2).
template <typename real>
__host__ __device__ __forceinline__ Prim<real> cons_to_prim(real r, real mx, real my, real mz, real E,
                                                   real gm1) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<real, float>::value) {
    // one reciprocal for the three velocities, paired products
    const float ir = q_div(1.0f, r);
    const float2 vxy = p_mul(f2(mx, my), f2s(ir));
    const float vz = mz * ir;
    const float2 sq = p_mul(vxy, vxy);
    const float v2 = rfma(vz, vz, radd(sq.x, sq.y));
    return Prim<float>{r, vxy.x, vxy.y, vz, rmul(gm1, rfma(rmul(-0.5f, r), v2, E))};
  }
#endif
  Prim<real> w;
  w.r = r;
  w.vx = q_div(mx, r);
  w.vy = q_div(my, r);
  w.vz = q_div(mz, r);
  const real v2 = rfma(w.vz, w.vz, rfma(w.vy, w.vy, rmul(w.vx, w.vx)));
  w.p = rmul(gm1, rfma(rmul(real(-0.5), r), v2, E));
  return w;
}

// MC(a, b) = 0 if a*b <= 0 else sign(a) min(2|a|, 2|b|, |a+b|/2)  (App. A.1, MC limiter).
template <typename real>
__host__ __device__ __forceinline__ real mc_slope(real a, real b) {
  real m = fmin(fmin(real(2) * fabs(a), real(2) * fabs(b)), real(0.5) * fabs(a + b));
  return (a * b > real(0)) ? copysign(m, a) : real(0);
}

// mc_slope on two lanes.  2 min(|a|, |b|, |a+b|/4) equals min(2|a|, 2|b|, |a+b|/2) bit for bit:
// scaling by powers of two is exact and commutes with min and |.|.
__device__ __forceinline__ float2 mc_slope2(float2 a, float2 b) {
  const float2 q = p_mul(p_add(a, b), f2s(0.25f));
  const float2 ab = p_mul(a, b);
  const float2 m = p_mul(f2(fminf(fminf(fabsf(a.x), fabsf(b.x)), fabsf(q.x)),
                            fminf(fminf(fabsf(a.y), fabsf(b.y)), fabsf(q.y))),
                         f2s(2.0f));
  return f2(ab.x > 0.0f ? copysignf(m.x, a.x) : 0.0f, ab.y > 0.0f ? copysignf(m.y, a.y) : 0.0f);
}

// Van Leer (App. A.1): 0 if a*b <= 0 else 2ab/(a+b), the harmonic form.
template <typename real>
__host__ __device__ __forceinline__ real vl_slope(real a, real b) {
  const real ab = a * b;
  return ab > real(0) ? q_div(real(2) * ab, a + b) : real(0);
}

// Slope limiters: LIM_MC (default) or LIM_VL.
constexpr int LIM_MC = 0, LIM_VL = 1;
template <int LIM, typename real>
__host__ __device__ __forceinline__ real lim_slope(real a, real b) {
  if constexpr (LIM == LIM_VL) return vl_slope(a, b);
  else return mc_slope(a, b);
}

// Limited slope of a cell from its two neighbours along one axis, with the positivity fallback:
// if W +- dW/2 has rho <= 0 or P <= 0 every slope of the cell on that axis is zero, and
// `fallbacks` is incremented.
template <int LIM = LIM_MC, typename real>
__host__ __device__ __forceinline__ Prim<real> limited_slope(const Prim<real>& wm, const Prim<real>& w0,
                                                    const Prim<real>& wp, int& fallbacks) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<real, float>::value && LIM == LIM_MC) {
    const float2 c01 = f2(w0.r, w0.vx), c23 = f2(w0.vy, w0.vz);
    const float2 d01 = mc_slope2(p_sub(f2(wp.r, wp.vx), c01), p_sub(c01, f2(wm.r, wm.vx)));
    const float2 d23 = mc_slope2(p_sub(f2(wp.vy, wp.vz), c23), p_sub(c23, f2(wm.vy, wm.vz)));
    const float dp = mc_slope(wp.p - w0.p, w0.p - wm.p);
    const float2 h = p_mul(f2(d01.x, dp), f2s(0.5f));        // half slopes of rho and P
    const float2 rp = f2(w0.r, w0.p);
    const float2 up = p_add(rp, h), dn = p_sub(rp, h);
    const bool bad = (up.x <= 0.0f) || (up.y <= 0.0f) || (dn.x <= 0.0f) || (dn.y <= 0.0f);
    if (bad) {
      ++fallbacks;
      return Prim<float>{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    }
    return Prim<float>{d01.x, d01.y, d23.x, d23.y, dp};
  }
#endif
  Prim<real> d;
  d.r = lim_slope<LIM>(wp.r - w0.r, w0.r - wm.r);
  d.vx = lim_slope<LIM>(wp.vx - w0.vx, w0.vx - wm.vx);
  d.vy = lim_slope<LIM>(wp.vy - w0.vy, w0.vy - wm.vy);
  d.vz = lim_slope<LIM>(wp.vz - w0.vz, w0.vz - wm.vz);
  d.p = lim_slope<LIM>(wp.p - w0.p, w0.p - wm.p);
  const real hr = real(0.5) * d.r, hp = real(0.5) * d.p;
  const bool bad = (w0.r + hr <= real(0)) || (w0.p + hp <= real(0)) || (w0.r - hr <= real(0)) ||
                   (w0.p - hp <= real(0));
  if (bad) {
    ++fallbacks;
    d = Prim<real>{real(0), real(0), real(0), real(0), real(0)};
  }
  return d;
}

template <int LIM = LIM_MC, typename real>
__host__ __device__ __forceinline__ Prim<real> limited_slope(const Prim<real>& wm, const Prim<real>& w0,
                                                    const Prim<real>& wp) {
  int unused = 0;
  return limited_slope<LIM>(wm, w0, wp, unused);
}

template <typename real>
__host__ __device__ __forceinline__ Prim<real> add_half(const Prim<real>& w, const Prim<real>& d, real s) {
  // w + s * d / 2 with s = +1 (left state of the upper face) or -1 (right state of the lower face)
  const real h = real(0.5) * s;
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<real, float>::value) {
    const float2 a = p_fma(f2(d.r, d.vx), f2s(h), f2(w.r, w.vx));
    const float2 b = p_fma(f2(d.vy, d.vz), f2s(h), f2(w.vy, w.vz));
    return Prim<float>{a.x, a.y, b.x, b.y, w.p + h * d.p};
  }
#endif
  return Prim<real>{w.r + h * d.r, w.vx + h * d.vx, w.vy + h * d.vy, w.vz + h * d.vz,
                    w.p + h * d.p};
}

// Flux components in the face frame: (mass, normal momentum, tangential 1, tangential 2, energy).
template <typename real> struct Flux { real f0, fn, ft1, ft2, fe; };

// Numerator and denominator of the contact speed S* (App. A.2):
// S* = (p_R - p_L + rho_L u_L d_L - rho_R u_R d_R) / (rho_L d_L - rho_R d_R), d_K = S_K - u_K.
// The flux and its adjoint both take these, so that they choose the same HLLC region.
template <typename real>
__host__ __device__ __forceinline__ real hllc_star_num(real rL, real uL, real pL, real dL, real rR,
                                                       real uR, real pR, real dR) {
  return rfma(-rmul(rR, uR), dR, rfma(rmul(rL, uL), dL, radd(pR, -pL)));
}
template <typename real>
__host__ __device__ __forceinline__ real hllc_star_den(real rL, real dL, real rR, real dR) {
  return rfma(rL, dL, -rmul(rR, dR));
}

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
  const real Sstar = q_div(hllc_star_num(rL, uL, pL, dL, rR, uR, pR, dR), hllc_star_den(rL, dL, rR, dR));

  // Select the side K whose (star) flux is taken.
  const bool left = (SL >= real(0)) || (Sstar >= real(0));
  const bool star = !(SL >= real(0)) && (Sstar >= real(0) || SR > real(0));
  const real r = left ? rL : rR, u = left ? uL : uR, a = left ? aL : aR, b = left ? bL : bR;
  const real p = left ? pL : pR, S = left ? SL : SR, d = left ? dL : dR;

  const real v2 = rfma(b, b, rfma(a, a, rmul(u, u)));
  const real E = rfma(rmul(real(0.5), r), v2, q_div(p, gm1));
  const real mass = rmul(r, u);
  Flux<real> F{mass, rfma(mass, u, p), rmul(mass, a), rmul(mass, b), rmul(u, radd(E, p))};
  if (star) {
    const real coef = q_div(rmul(r, d), radd(S, -Sstar));
    const real sdu = radd(Sstar, -u);
    const real Es = rmul(coef, rfma(sdu, radd(Sstar, q_div(p, rmul(r, d))), q_div(E, r)));
    F.f0 = rfma(S, radd(coef, -r), F.f0);
    F.fn = rfma(S, rfma(coef, Sstar, -mass), F.fn);
    F.ft1 = rfma(S, radd(rmul(coef, a), -rmul(r, a)), F.ft1);
    F.ft2 = rfma(S, radd(rmul(coef, b), -rmul(r, b)), F.ft2);
    F.fe = rfma(S, radd(Es, -E), F.fe);
  }
  return F;
}

// hllc() for float32 with the left and right states in the two lanes of packed operations.
__device__ __forceinline__ Flux<float> hllc_packed(float rL, float uL, float aL, float bL, float pL,
                                                   float rR, float uR, float aR, float bR, float pR,
                                                   float gamma, float gm1) {
  const float2 r = f2(rL, rR), u = f2(uL, uR), pp = f2(pL, pR);
  const float2 gp = p_mul(pp, f2s(gamma));
  // c = sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one reciprocal square root per side
  const float2 gpr = p_mul(gp, r);
  const float2 c = p_mul(gp, f2(gpr.x > 0.0f ? rsqrtf(gpr.x) : 0.0f, gpr.y > 0.0f ? rsqrtf(gpr.y) : 0.0f));
  const float2 um = p_sub(u, c), upc = p_add(u, c);
  const float SL = fminf(um.x, um.y);
  const float SR = fmaxf(upc.x, upc.y);
  const float2 d = p_sub(f2(SL, SR), u);            // (S_L - u_L, S_R - u_R)
  const float2 rd = p_mul(r, d);
  // numerator p_R - p_L + rho_L u_L d_L - rho_R u_R d_R as (rd_L u_L - p_L) - (rd_R u_R - p_R)
  const float2 t = p_sub(p_mul(rd, u), pp);
  const float Sstar = q_div(t.x - t.y, rd.x - rd.y);

  const bool left = (SL >= 0.0f) || (Sstar >= 0.0f);
  const bool star = !(SL >= 0.0f) && (Sstar >= 0.0f || SR > 0.0f);
  const float rk = left ? rL : rR, uk = left ? uL : uR, ak = left ? aL : aR, bk = left ? bL : bR;
  const float pk = left ? pL : pR, S = left ? SL : SR, dk = left ? d.x : d.y;

  const float2 ua2 = p_mul(f2(uk, ak), f2(uk, ak));
  const float igm1 = 1.0f / gm1;   // uniform: hoisted out of the face loops
  const float E = rfma(pk, igm1, rmul(rmul(0.5f, rk), rfma(bk, bk, radd(ua2.x, ua2.y))));
  const float mass = rmul(rk, uk);
  const float2 fna = p_fma(f2s(mass), f2(uk, ak), f2(pk, 0.0f));   // (mass u + p, mass a)
  Flux<float> F{mass, fna.x, fna.y, rmul(mass, bk), rmul(uk, radd(E, pk))};
  if (star) {
    // E* = rho d/(S - S*) (E/rho + (S* - u)(S* + p/(rho d))) with one reciprocal:
    // = (d (E + rho S* (S* - u)) + (S* - u) p) / (S - S*)
    const float inv = q_div(1.0f, radd(S, -Sstar));
    const float rdk = rmul(rk, dk);
    const float coef = rmul(rdk, inv);
    const float sdu = radd(Sstar, -uk);
    const float Es = rmul(rfma(dk, rfma(rmul(rk, Sstar), sdu, E), rmul(sdu, pk)), inv);
    const float w = radd(coef, -rk);
    const float2 f0n = p_fma(f2s(S), f2(w, rfma(coef, Sstar, -mass)), f2(F.f0, F.fn));
    const float2 ft = p_fma(f2s(rmul(S, w)), f2(ak, bk), f2(F.ft1, F.ft2));
    F.f0 = f0n.x;
    F.fn = f0n.y;
    F.ft1 = ft.x;
    F.ft2 = ft.y;
    F.fe = rfma(S, radd(Es, -E), F.fe);
  }
  return F;
}

// HLLC flux across a face normal to `axis` (0 = x, 1 = y, 2 = z) from reconstructed
// primitive states; returns fluxes in (rho, m_x, m_y, m_z, E) order.
template <typename real>
__host__ __device__ __forceinline__ void face_flux(int axis, const Prim<real>& L, const Prim<real>& R,
                                          real gamma, real gm1, real out[5]) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<real, float>::value) {
    if (axis == 0) {
      Flux<float> F = hllc_packed(L.r, L.vx, L.vy, L.vz, L.p, R.r, R.vx, R.vy, R.vz, R.p, gamma, gm1);
      out[0] = F.f0; out[1] = F.fn; out[2] = F.ft1; out[3] = F.ft2; out[4] = F.fe;
    } else if (axis == 1) {
      Flux<float> F = hllc_packed(L.r, L.vy, L.vx, L.vz, L.p, R.r, R.vy, R.vx, R.vz, R.p, gamma, gm1);
      out[0] = F.f0; out[1] = F.ft1; out[2] = F.fn; out[3] = F.ft2; out[4] = F.fe;
    } else {
      Flux<float> F = hllc_packed(L.r, L.vz, L.vx, L.vy, L.p, R.r, R.vz, R.vx, R.vy, R.p, gamma, gm1);
      out[0] = F.f0; out[1] = F.ft1; out[2] = F.ft2; out[3] = F.fn; out[4] = F.fe;
    }
    return;
  }
#endif
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
