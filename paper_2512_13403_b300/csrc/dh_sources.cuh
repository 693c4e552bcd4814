// Per-cell source terms shared by the fused stage-2 epilogue and the gravity-path source kernel:
// OU forcing synthesis (Sec. 3.1.1), optically thin cooling (Sec. 4.3) and the CFL time of a
// cell (App. A.4).
#pragma once
#include <type_traits>

#include "dh_device.cuh"
#include "ff.cuh"

namespace dh {

// g = -grad phi by central differences (Sec. 5) from the float-float potential (planar, n hi
// words then n lo words; grids below 2^31 cells).  For a float32 result the two words are
// differenced separately: hi - hi is exact when the two lie within a factor 2 of each other
// (Sterbenz) and otherwise rounds below an ulp of the result, so the float-float difference is
// not needed.  For float64 the difference is taken in float-float.
//
// The 12 float-float words of the potential that g = -grad phi at cell (i, j, k) needs:
// (hi, lo) of the +x, -x, +y, -y, +z, -z neighbours (periodic).
__device__ __forceinline__ void potential_gradient_load(const float* __restrict__ phi, int nx, int ny,
                                                        int nz, int i, int j, int k, float v[12]) {
  const unsigned plane = (unsigned)nx * (unsigned)ny, n = plane * (unsigned)nz;
  const unsigned q = ((unsigned)k * (unsigned)ny + (unsigned)j) * (unsigned)nx + (unsigned)i;
  const unsigned xm = i == 0 ? q + nx - 1 : q - 1, xp = i == nx - 1 ? q + 1 - nx : q + 1;
  const unsigned ym = j == 0 ? q + plane - nx : q - nx, yp = j == ny - 1 ? q + nx - plane : q + nx;
  const unsigned zm = k == 0 ? q + n - plane : q - plane, zp = k == nz - 1 ? q + plane - n : q + plane;
  const float* __restrict__ lo = phi + n;
  v[0] = phi[xp]; v[1] = lo[xp]; v[2] = phi[xm]; v[3] = lo[xm];
  v[4] = phi[yp]; v[5] = lo[yp]; v[6] = phi[ym]; v[7] = lo[ym];
  v[8] = phi[zp]; v[9] = lo[zp]; v[10] = phi[zm]; v[11] = lo[zm];
}

// g from the words of potential_gradient_load.
template <typename real>
__device__ __forceinline__ void potential_gradient_eval(const float v[12], real i2h, real& g0,
                                                        real& g1, real& g2) {
  if constexpr (std::is_same<real, float>::value) {
    g0 = -((v[0] - v[2]) + (v[1] - v[3])) * i2h;
    g1 = -((v[4] - v[6]) + (v[5] - v[7])) * i2h;
    g2 = -((v[8] - v[10]) + (v[9] - v[11])) * i2h;
  } else {
    const ff2 dx = ff_sub(ff2{v[0], v[1]}, ff2{v[2], v[3]});
    const ff2 dy = ff_sub(ff2{v[4], v[5]}, ff2{v[6], v[7]});
    const ff2 dz = ff_sub(ff2{v[8], v[9]}, ff2{v[10], v[11]});
    g0 = -((real)dx.hi + (real)dx.lo) * i2h;
    g1 = -((real)dy.hi + (real)dy.lo) * i2h;
    g2 = -((real)dz.hi + (real)dz.lo) * i2h;
  }
}

template <typename real>
__device__ __forceinline__ void potential_gradient(const float* __restrict__ phi, int nx, int ny,
                                                   int nz, int i, int j, int k, real i2h, real& g0,
                                                   real& g1, real& g2) {
  float v[12];
  potential_gradient_load(phi, nx, ny, nz, i, j, k, v);
  potential_gradient_eval(v, i2h, g0, g1, g2);
}

// Forced-mode table of Sec. 3.1.1 as compile-time data: the half-space of integer n with
// 1 <= |n|^2 <= 4 whose first nonzero component is positive, lexicographic in (n_x, n_y, n_z).
__host__ __device__ constexpr int forced_mode_component(int m, int axis) {
  int count = 0;
  for (int a = -2; a <= 2; ++a)
    for (int b = -2; b <= 2; ++b)
      for (int c = -2; c <= 2; ++c) {
        const int k2 = a * a + b * b + c * c;
        const int first = a != 0 ? a : (b != 0 ? b : c);
        if (k2 >= 1 && k2 <= 4 && first > 0) {
          if (count == m) return axis == 0 ? a : (axis == 1 ? b : c);
          ++count;
        }
      }
  return 0;
}
static_assert(forced_mode_component(15, 0) == 2 && forced_mode_component(0, 2) == 1,
              "forced mode enumeration");

template <typename real> struct C2 { real re, im; };

template <typename real>
__device__ __forceinline__ C2<real> cmul(C2<real> a, C2<real> b) {
  return C2<real>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// exp(2 pi i n x~) for one axis from its twiddles (n in -2..2, n != 0).
template <typename real, int N>
__device__ __forceinline__ C2<real> axis_factor(const real* t) {
  static_assert(N != 0, "");
  constexpr int A = N > 0 ? N : -N;
  const real c = A == 1 ? t[0] : t[2];
  const real s = A == 1 ? t[1] : t[3];
  return C2<real>{c, N > 0 ? s : -s};
}

template <typename real, int M>
__device__ __forceinline__ void add_mode(const real* __restrict__ ah, const real* tx,
                                         const real* ty, const real* tz, real acc[3]) {
  constexpr int NX = forced_mode_component(M, 0);
  constexpr int NY = forced_mode_component(M, 1);
  constexpr int NZ = forced_mode_component(M, 2);
  C2<real> e{real(1), real(0)};
  bool first = true;
  if constexpr (NX != 0) { e = axis_factor<real, NX>(tx); first = false; }
  if constexpr (NY != 0) {
    const C2<real> f = axis_factor<real, NY>(ty);
    e = first ? f : cmul(e, f);
    first = false;
  }
  if constexpr (NZ != 0) {
    const C2<real> f = axis_factor<real, NZ>(tz);
    e = first ? f : cmul(e, f);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const real are = __ldg(ah + 2 * (3 * M + c));
    const real aim = __ldg(ah + 2 * (3 * M + c) + 1);
    acc[c] += are * e.re - aim * e.im;
  }
}

template <typename real, int M>
__device__ __forceinline__ void add_modes(const real* ah, const real* tx, const real* ty,
                                          const real* tz, real acc[3]) {
  if constexpr (M < 16) {
    add_mode<real, M>(ah, tx, ty, tz, acc);
    add_modes<real, M + 1>(ah, tx, ty, tz, acc);
  }
}

// One task of the per-row forcing factors: for row (y, z) and n_x in {0,1,2}, component c:
// B = sum over forced modes with that n_x of a_hat_{m,c} exp(2 pi i (n_y y~ + n_z z~)).
// `ah` (the normalised table) may be in global or shared memory.
template <typename real, int M>
__device__ __forceinline__ void row_factor(const real* __restrict__ ah, int nxsel, int c,
                                           const real* ty, const real* tz, real& bre, real& bim) {
  if constexpr (M < 16) {
    constexpr int NX = forced_mode_component(M, 0);
    constexpr int NY = forced_mode_component(M, 1);
    constexpr int NZ = forced_mode_component(M, 2);
    if (NX == nxsel) {
      C2<real> e{real(1), real(0)};
      bool first = true;
      if constexpr (NY != 0) { e = axis_factor<real, NY>(ty); first = false; }
      if constexpr (NZ != 0) {
        const C2<real> f = axis_factor<real, NZ>(tz);
        e = first ? f : cmul(e, f);
      }
      const real are = ah[2 * (3 * M + c)];
      const real aim = ah[2 * (3 * M + c) + 1];
      bre += are * e.re - aim * e.im;
      bim += are * e.im + aim * e.re;
    }
    row_factor<real, M + 1>(ah, nxsel, c, ty, tz, bre, bim);
  }
}

// The row factors of all three n_x bins for row (y, z) and component c at once: bin b collects
// the modes with n_x = b, in the mode order of row_factor.
template <typename real, int M>
__device__ __forceinline__ void row_factors3(const real* __restrict__ ah, int c, const real* ty,
                                             const real* tz, real bre[3], real bim[3]) {
  if constexpr (M < 16) {
    constexpr int NX = forced_mode_component(M, 0);
    constexpr int NY = forced_mode_component(M, 1);
    constexpr int NZ = forced_mode_component(M, 2);
    C2<real> e{real(1), real(0)};
    bool first = true;
    if constexpr (NY != 0) { e = axis_factor<real, NY>(ty); first = false; }
    if constexpr (NZ != 0) {
      const C2<real> f = axis_factor<real, NZ>(tz);
      e = first ? f : cmul(e, f);
    }
    const real are = ah[2 * (3 * M + c)];
    const real aim = ah[2 * (3 * M + c) + 1];
    bre[NX] += are * e.re - aim * e.im;
    bim[NX] += are * e.im + aim * e.re;
    row_factors3<real, M + 1>(ah, c, ty, tz, bre, bim);
  }
}

// a(x) = 2 Re sum_H a_hat_n exp(2 pi i n . x~), with the normalised table (Sec. 3.1.1).
template <typename real>
__device__ __forceinline__ void forcing_accel(const real* ah, const real* const tw[3], int i,
                                              int j, int k, real a[3]) {
  real tx[4], ty[4], tz[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    tx[q] = __ldg(tw[0] + 4 * i + q);
    ty[q] = __ldg(tw[1] + 4 * j + q);
    tz[q] = __ldg(tw[2] + 4 * k + q);
  }
  real acc[3] = {real(0), real(0), real(0)};
  add_modes<real, 0>(ah, tx, ty, tz, acc);
  a[0] = real(2) * acc[0];
  a[1] = real(2) * acc[1];
  a[2] = real(2) * acc[2];
}

// Cooling of one cell (Sec. 4.3; Lambda = n^2 T^(1/2), T = P / rho, floor rho T_floor/(gamma-1)).
// A cell cools only while its thermal energy is above the floor energy; the test compares
// energies, so a state clamped to the floor is recognised exactly whatever the rounding of T.
// Products, sums and fused multiply-adds have their rounding spelled out (never contracted by
// the compiler), so the two-lane form (cooling_energy2) and the tangents (cooling_tangents)
// take exactly this function's values and branches.
template <typename real>
__device__ __forceinline__ real cooling_rate(real r2, real gm1, real Eth, real ir) {
  return -rmul(r2, q_sqrt(rmul(rmul(gm1, Eth), ir)));
}
template <typename real>
__device__ __forceinline__ real cooling_energy(real r, real mx, real my, real mz, real E, real dt,
                                               real gm1, real T_floor, real frac, int nsub_max,
                                               unsigned& flags, int& nsub_seen) {
  const real ir = q_div(real(1), r);
  const real kin = rmul(rmul(real(0.5), rfma(mz, mz, rfma(my, my, rmul(mx, mx)))), ir);
  const real Eth = radd(E, -kin);
  const real Efl = rmul(rmul(r, T_floor), real(1) / gm1);
  if (!(Eth > Efl)) return E;
  const real r2 = rmul(r, r);
  const real Ed0 = cooling_rate(r2, gm1, Eth, ir);
  // dt / (frac t_cool) with t_cool = Eth / (-Ed0), as one division
  const real raw = ceil(q_div(rmul(dt, -Ed0), rmul(frac, Eth)));
  // clamp to [1, nsub_max]; a NaN count also takes the cap, so the loop below is always bounded
  real nsub = raw;
  if (!(raw <= real(nsub_max))) {
    if (raw > real(nsub_max)) flags |= FLAG_COOL_CAP;
    nsub = real(nsub_max);
  }
  if (!(nsub >= real(1))) nsub = real(1);
  real Enew;
  if (nsub == real(1)) {
    const real Ep = fmax(Efl, rfma(dt, Ed0, Eth));
    const real Edp = Ep > Efl ? cooling_rate(r2, gm1, Ep, ir) : real(0);
    Enew = fmax(Efl, rfma(real(0.5) * dt, radd(Ed0, Edp), Eth));
  } else {
    const real dts = q_div(dt, nsub);
    const int n = (int)nsub;
    nsub_seen = n > nsub_seen ? n : nsub_seen;
    real Es = Eth;
    for (int q = 0; q < n; ++q) {
      const real ed = Es > Efl ? cooling_rate(r2, gm1, Es, ir) : real(0);
      Es = fmax(Efl, rfma(ed, dts, Es));
    }
    Enew = Es;
  }
  return radd(kin, Enew);
}

// Tangents of the cooling map of one cell, (rho, E_th) -> E_th', as cooling_energy computes it:
// cR = dE_th'/drho at fixed E_th, cE = dE_th'/dE_th.  Forward-mode along the same branches and
// substeps; the substep count is a frozen integer.  Rules: a clamp max(E_floor, X) takes the
// tangent of the larger argument (half of each on an exact tie); the rate -rho^2 sqrt(T),
// T = (gamma-1) E / rho, has d(rate) = 1.5 rate/rho drho + 0.5 rate/E dE above the floor and is
// zero at or below it.  A cell that does not cool is the identity (cR = 0, cE = 1).
template <typename real>
__device__ __forceinline__ void cooling_tangents(real r, real mx, real my, real mz, real E, real dt,
                                                 real gm1, real T_floor, real frac, int nsub_max,
                                                 real& cR, real& cE) {
  const real ir = q_div(real(1), r);
  const real kin = rmul(rmul(real(0.5), rfma(mz, mz, rfma(my, my, rmul(mx, mx)))), ir);
  const real Eth = radd(E, -kin);
  const real Efl = rmul(rmul(r, T_floor), real(1) / gm1);
  cR = real(0);
  cE = real(1);
  if (!(Eth > Efl)) return;
  const real dfl = q_div(T_floor, gm1);   // dE_floor/drho
  const real r2 = rmul(r, r);
  // clamp rule for max(E_floor, X) with tangent (xr, xe)
  auto clamp_t = [&](real X, real xr, real xe, real& tr, real& te) {
    if (X > Efl) { tr = xr; te = xe; }
    else if (X < Efl) { tr = dfl; te = real(0); }
    else { tr = real(0.5) * (xr + dfl); te = real(0.5) * xe; }
  };
  const real Ed0 = cooling_rate(r2, gm1, Eth, ir);
  const real raw = ceil(q_div(rmul(dt, -Ed0), rmul(frac, Eth)));   // the forward's substep count
  real nsub = raw;
  if (!(raw <= real(nsub_max))) nsub = real(nsub_max);
  if (!(nsub >= real(1))) nsub = real(1);
  if (nsub == real(1)) {
    const real d0r = real(1.5) * Ed0 * ir, d0e = real(0.5) * q_div(Ed0, Eth);
    const real X = rfma(dt, Ed0, Eth);
    real pr, pe;
    clamp_t(X, dt * d0r, real(1) + dt * d0e, pr, pe);
    const real Ep = fmax(Efl, X);
    real Edp = real(0), dpr = real(0), dpe = real(0);
    if (Ep > Efl) {
      Edp = cooling_rate(r2, gm1, Ep, ir);
      const real g = real(0.5) * q_div(Edp, Ep);
      dpr = real(1.5) * Edp * ir + g * pr;
      dpe = g * pe;
    }
    const real Y = rfma(real(0.5) * dt, radd(Ed0, Edp), Eth);
    clamp_t(Y, real(0.5) * dt * (d0r + dpr), real(1) + real(0.5) * dt * (d0e + dpe), cR, cE);
  } else {
    const real dts = q_div(dt, nsub);
    const int n = (int)nsub;
    real Es = Eth, sr = real(0), se = real(1);
    for (int q = 0; q < n; ++q) {
      real ed = real(0), er = real(0), ee = real(0);
      if (Es > Efl) {
        ed = cooling_rate(r2, gm1, Es, ir);
        const real g = real(0.5) * q_div(ed, Es);
        er = real(1.5) * ed * ir + g * sr;
        ee = g * se;
      }
      const real X = rfma(ed, dts, Es);
      real tr, te;
      clamp_t(X, sr + dts * er, se + dts * ee, tr, te);
      Es = fmax(Efl, X);
      sr = tr;
      se = te;
    }
    cR = sr;
    cE = se;
  }
}

// Cooling time t_cool = E_th / |Edot| = E_th / (rho^2 T^(1/2)) of a cell above the floor energy
// (Sec. 4.3), +inf at or below it (where nothing cools).
template <typename real>
__device__ __forceinline__ real cooling_time(real r, real mx, real my, real mz, real E, real gm1,
                                             real T_floor) {
  const real ir = q_div(real(1), r);
  const real Eth = E - real(0.5) * (mx * mx + my * my + mz * mz) * ir;
  const real Efl = r * T_floor * (real(1) / gm1);
  if (!(Eth > Efl)) return real(INFINITY);
  return q_div(Eth, r * r * q_sqrt(gm1 * Eth * ir));
}

template <typename real>
__device__ __forceinline__ real cfl_time(real r, real mx, real my, real mz, real E, real gamma,
                                         real gm1, real dx, real dy, real dz) {
  const Prim<real> w = cons_to_prim(r, mx, my, mz, E, gm1);
  real c;
  if constexpr (std::is_same<real, float>::value) {
    const float gpr = gamma * w.p * w.r;    // c = gamma p / sqrt(gamma p rho)
    c = gpr > 0.0f ? gamma * w.p * rsqrtf(gpr) : 0.0f;
  } else {
    c = q_sqrt(q_div(gamma * w.p, w.r));
  }
  const real tx = q_div(dx, fabs(w.vx) + c);
  const real ty = q_div(dy, fabs(w.vy) + c);
  const real tz = q_div(dz, fabs(w.vz) + c);
  return fmin(fmin(tx, ty), tz);
}

}  // namespace dh
