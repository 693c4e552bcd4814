// Two-cell lanes for the paired stage kernel (hydro_pair.cu): every quantity of the finite-volume
// update (App. A.1-A.3) is carried for two cells at once, lane x for cell A and lane y for cell
// B.  For float32 the lanes are the two halves of the packed FADD2/FMUL2/FFMA2 instructions of
// sm_100+, so a pair costs one arithmetic instruction and no register shuffling (both lanes of
// every value already sit in one register pair); for float64 each lane is a scalar operation.
// Every operation rounds each lane once (IEEE round to nearest, no contraction), so a cell's
// result does not depend on its lane.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dh_device.cuh"

namespace dh {

template <typename real> struct PairOf;
template <> struct PairOf<float> { using T = float2; };
template <> struct PairOf<double> { using T = double2; };
template <typename real> using pair_t = typename PairOf<real>::T;

// Four reals: the pairs of two fields side by side (one 16-byte shared-memory access for float).
template <typename real> struct alignas(4 * sizeof(real) > 16 ? 16 : 4 * sizeof(real)) Quad {
  pair_t<real> a, b;
};

__device__ __forceinline__ float2 pset(float s) { return make_float2(s, s); }
__device__ __forceinline__ double2 pset(double s) { return make_double2(s, s); }
__device__ __forceinline__ float2 pmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pmk(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b: fma(b, -1, a) rounds the exact difference once
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, pset(-1.0f), a); }

__device__ __forceinline__ double2 padd(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
  return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) {
  return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}

template <typename P> __device__ __forceinline__ P pmin(P a, P b) { return pmk(fmin(a.x, b.x), fmin(a.y, b.y)); }
template <typename P> __device__ __forceinline__ P pmax(P a, P b) { return pmk(fmax(a.x, b.x), fmax(a.y, b.y)); }
template <typename P> __device__ __forceinline__ P pneg(P a) { return pmk(-a.x, -a.y); }

// Lane-wise quotient and reciprocal: q_div of the working precision (the float32 hardware
// reciprocal, IEEE division in float64).
template <typename P> __device__ __forceinline__ P pdiv(P a, P b) { return pmk(q_div(a.x, b.x), q_div(a.y, b.y)); }

// Primitive state of two cells.
template <typename real> struct Prim2 { pair_t<real> r, vx, vy, vz, p; };

// W = (rho, v, P) of two cells from their conserved variables (Eq. 2): one reciprocal of rho
// per lane, P = (gamma - 1)(E - rho |v|^2 / 2).
template <typename real>
__device__ __forceinline__ Prim2<real> cons_to_prim2(pair_t<real> r, pair_t<real> mx, pair_t<real> my,
                                                     pair_t<real> mz, pair_t<real> E, real gm1) {
  using P = pair_t<real>;
  const P ir = pdiv(pset(real(1)), r);
  Prim2<real> w;
  w.r = r;
  w.vx = pmul(mx, ir);
  w.vy = pmul(my, ir);
  w.vz = pmul(mz, ir);
  const P v2 = pfma(w.vz, w.vz, pfma(w.vy, w.vy, pmul(w.vx, w.vx)));
  w.p = pmul(pset(gm1), pfma(pmul(pset(real(-0.5)), r), v2, E));
  return w;
}

// Half of the limited slope, dW/2, of one field for two cells from the forward and backward
// differences a = W_{i+1} - W_i, b = W_i - W_{i-1} (App. A.1).
//   MC: dW = 0 if ab <= 0, else sign(a) min(2|a|, 2|b|, |a+b|/2), so dW/2 = sign(a) min(|a|, |b|, |a+b|/4)
//   van Leer: dW = 0 if ab <= 0, else 2ab/(a+b), so dW/2 = ab/(a+b)
// Halving is exact, so W +- dW/2 has the bits of W +- (1/2) dW.
template <int LIM, typename P>
__device__ __forceinline__ P half_slope2(P a, P b) {
  const P ab = pmul(a, b);
  if constexpr (LIM == LIM_VL) {
    const P h = pdiv(ab, padd(a, b));
    return pmk(ab.x > 0 ? h.x : decltype(h.x)(0), ab.y > 0 ? h.y : decltype(h.y)(0));
  } else {
    using R = decltype(a.x);
    const P q = pmul(padd(a, b), pset(R(0.25)));
    const R mx = fmin(fmin(fabs(a.x), fabs(b.x)), fabs(q.x));
    const R my = fmin(fmin(fabs(a.y), fabs(b.y)), fabs(q.y));
    return pmk(ab.x > R(0) ? copysign(mx, a.x) : R(0), ab.y > R(0) ? copysign(my, a.y) : R(0));
  }
}

// Half slopes of all five primitives of two cells along one axis from the cell (w0) and its two
// neighbours, with the positivity fallback: a lane whose face states W +- dW/2 have rho <= 0 or
// P <= 0 takes zero slopes on this axis (first order) and adds one to its count.
template <int LIM, typename real>
__device__ __forceinline__ Prim2<real> limited_half2(const Prim2<real>& wm, const Prim2<real>& w0,
                                                     const Prim2<real>& wp, int& nfa, int& nfb) {
  using P = pair_t<real>;
  Prim2<real> h;
  h.r = half_slope2<LIM>(psub(wp.r, w0.r), psub(w0.r, wm.r));
  h.vx = half_slope2<LIM>(psub(wp.vx, w0.vx), psub(w0.vx, wm.vx));
  h.vy = half_slope2<LIM>(psub(wp.vy, w0.vy), psub(w0.vy, wm.vy));
  h.vz = half_slope2<LIM>(psub(wp.vz, w0.vz), psub(w0.vz, wm.vz));
  h.p = half_slope2<LIM>(psub(wp.p, w0.p), psub(w0.p, wm.p));
  const P ru = padd(w0.r, h.r), rd = psub(w0.r, h.r);
  const P pu = padd(w0.p, h.p), pd = psub(w0.p, h.p);
  const bool bx = (ru.x <= real(0)) || (rd.x <= real(0)) || (pu.x <= real(0)) || (pd.x <= real(0));
  const bool by = (ru.y <= real(0)) || (rd.y <= real(0)) || (pu.y <= real(0)) || (pd.y <= real(0));
  if (bx || by) {
    nfa += bx ? 1 : 0;
    nfb += by ? 1 : 0;
    auto z = [&](P& v) { v = pmk(bx ? real(0) : v.x, by ? real(0) : v.y); };
    z(h.r); z(h.vx); z(h.vy); z(h.vz); z(h.p);
  }
  return h;
}

// W + s dW/2 for s = +1 (left state of the upper face) or -1 (right state of the lower face).
template <typename real>
__device__ __forceinline__ Prim2<real> face_state2(const Prim2<real>& w, const Prim2<real>& h, bool upper) {
  if (upper)
    return Prim2<real>{padd(w.r, h.r), padd(w.vx, h.vx), padd(w.vy, h.vy), padd(w.vz, h.vz), padd(w.p, h.p)};
  return Prim2<real>{psub(w.r, h.r), psub(w.vx, h.vx), psub(w.vy, h.vy), psub(w.vz, h.vz), psub(w.p, h.p)};
}

// Sound speed c = sqrt(gamma p / rho) of two states: float32 takes gamma p / sqrt(gamma p rho)
// (one reciprocal square root per lane, zero for a non-positive argument), float64 the IEEE
// square root of the quotient.
template <typename real>
__device__ __forceinline__ pair_t<real> sound_speed2(pair_t<real> r, pair_t<real> p, real gamma) {
  if constexpr (std::is_same<real, float>::value) {
    const float2 gp = pmul(p, pset(gamma));
    const float2 gpr = pmul(gp, r);
    return pmul(gp, make_float2(gpr.x > 0.0f ? rsqrtf(gpr.x) : 0.0f, gpr.y > 0.0f ? rsqrtf(gpr.y) : 0.0f));
  } else {
    const double2 q = pdiv(pmul(p, pset(gamma)), r);
    return make_double2(sqrt(q.x), sqrt(q.y));
  }
}

// HLLC flux (Toro, Spruce & Speares; Davis wave speeds, App. A.2) of two faces, in the face
// frame (rho, u_n, u_t1, u_t2, P) for each side.  Region per lane: S_L >= 0 -> F_L;
// S* >= 0 -> F*_L; S_R > 0 -> F*_R; else F_R.  Output (mass, normal momentum, tangential 1,
// tangential 2, energy).  Lanes outside the star regions add S_eff = 0 times finite star terms
// (their denominator is replaced by 1), which leaves their flux unchanged.
template <typename real>
__device__ __forceinline__ void hllc2(const pair_t<real> rL, const pair_t<real> uL, const pair_t<real> aL,
                                      const pair_t<real> bL, const pair_t<real> pL, const pair_t<real> rR,
                                      const pair_t<real> uR, const pair_t<real> aR, const pair_t<real> bR,
                                      const pair_t<real> pR, real gamma, real igm1, pair_t<real> F[5]) {
  using P = pair_t<real>;
  const P cL = sound_speed2<real>(rL, pL, gamma), cR = sound_speed2<real>(rR, pR, gamma);
  const P SL = pmin(psub(uL, cL), psub(uR, cR));
  const P SR = pmax(padd(uL, cL), padd(uR, cR));
  const P dL = psub(SL, uL), dR = psub(SR, uR);
  const P rdL = pmul(rL, dL), rdR = pmul(rR, dR);
  // S* = ((rho_L d_L u_L - p_L) - (rho_R d_R u_R - p_R)) / (rho_L d_L - rho_R d_R)
  const P tL = psub(pmul(rdL, uL), pL), tR = psub(pmul(rdR, uR), pR);
  const P Ss = pdiv(psub(tL, tR), psub(rdL, rdR));

  bool left[2], star[2];
  left[0] = (SL.x >= real(0)) || (Ss.x >= real(0));
  left[1] = (SL.y >= real(0)) || (Ss.y >= real(0));
  star[0] = !(SL.x >= real(0)) && (Ss.x >= real(0) || SR.x > real(0));
  star[1] = !(SL.y >= real(0)) && (Ss.y >= real(0) || SR.y > real(0));
  auto sel = [&](P l, P r) { return pmk(left[0] ? l.x : r.x, left[1] ? l.y : r.y); };
  const P rk = sel(rL, rR), uk = sel(uL, uR), ak = sel(aL, aR), bk = sel(bL, bR);
  const P pk = sel(pL, pR), S = sel(SL, SR), dk = sel(dL, dR);

  const P E = pfma(pk, pset(igm1), pmul(pmul(pset(real(0.5)), rk), pfma(bk, bk, pfma(ak, ak, pmul(uk, uk)))));
  const P mass = pmul(rk, uk);
  P f0 = mass;
  P fn = pfma(mass, uk, pk);
  P ft1 = pmul(mass, ak);
  P ft2 = pmul(mass, bk);
  P fe = pmul(uk, padd(E, pk));
  if (star[0] || star[1]) {
    // E* = (d (E + rho S* (S* - u)) + (S* - u) p) / (S - S*)
    const P den = psub(S, Ss);
    const P inv = pdiv(pset(real(1)), pmk(star[0] ? den.x : real(1), star[1] ? den.y : real(1)));
    const P Se = pmk(star[0] ? S.x : real(0), star[1] ? S.y : real(0));
    const P coef = pmul(pmul(rk, dk), inv);
    const P sdu = psub(Ss, uk);
    const P Es = pmul(pfma(dk, pfma(pmul(rk, Ss), sdu, E), pmul(sdu, pk)), inv);
    const P w = psub(coef, rk);
    const P Sw = pmul(Se, w);
    f0 = pfma(Se, w, f0);
    fn = pfma(Se, pfma(coef, Ss, pneg(mass)), fn);
    ft1 = pfma(Sw, ak, ft1);
    ft2 = pfma(Sw, bk, ft2);
    fe = pfma(Se, psub(Es, E), fe);
  }
  F[0] = f0; F[1] = fn; F[2] = ft1; F[3] = ft2; F[4] = fe;
}

// HLLC flux of two faces normal to `AXIS` from the reconstructed primitive states, in
// (rho, m_x, m_y, m_z, E) order.
template <int AXIS, typename real>
__device__ __forceinline__ void face_flux2(const Prim2<real>& L, const Prim2<real>& R, real gamma, real igm1,
                                           pair_t<real> out[5]) {
  pair_t<real> F[5];
  if constexpr (AXIS == 0) {
    hllc2<real>(L.r, L.vx, L.vy, L.vz, L.p, R.r, R.vx, R.vy, R.vz, R.p, gamma, igm1, F);
    out[0] = F[0]; out[1] = F[1]; out[2] = F[2]; out[3] = F[3]; out[4] = F[4];
  } else if constexpr (AXIS == 1) {
    hllc2<real>(L.r, L.vy, L.vx, L.vz, L.p, R.r, R.vy, R.vx, R.vz, R.p, gamma, igm1, F);
    out[0] = F[0]; out[1] = F[2]; out[2] = F[1]; out[3] = F[3]; out[4] = F[4];
  } else {
    hllc2<real>(L.r, L.vz, L.vx, L.vy, L.p, R.r, R.vz, R.vx, R.vy, R.p, gamma, igm1, F);
    out[0] = F[0]; out[1] = F[2]; out[2] = F[3]; out[3] = F[1]; out[4] = F[4];
  }
}

}  // namespace dh
