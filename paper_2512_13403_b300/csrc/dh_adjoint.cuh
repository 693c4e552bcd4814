// Per-face reverse-mode building blocks of the hand adjoint: the MC and van Leer slopes, the
// limited slope with its positivity fallback, HLLC and the face VJP of HLLC on reconstructed
// states (App. A.1-A.2 transposed).  Host and device code; the GPU kernels that use them are
// checked against reverse-mode differentiation of the oracle step and against finite
// differences.
#pragma once
#include "dh_device.cuh"

namespace dh {

// Reverse of mc_slope for one component: D = dL/d(slope) -> (dL/da, dL/db).  Where a b > 0 the
// slope is sign(a) min(2|a|, 2|b|, |a+b|/2); its three branches have the derivatives (2, 0),
// (0, 2) and (1/2, 1/2) in (a, b), and a tie splits the derivative evenly between the tied
// branches.  Branch-free: the branch weights are 0, 1/2 or 1.
template <typename real>
__host__ __device__ __forceinline__ void mc_slope_vjp(real a, real b, real D, real& ga, real& gb) {
  const real X = real(2) * fabs(a), Y = real(2) * fabs(b), Z = real(0.5) * fabs(a + b);
  const real m1 = fmin(X, Y);
  const real wm = m1 < Z ? real(1) : (m1 == Z ? real(0.5) : real(0));   // weight of min(X, Y)
  const real wx = X < Y ? real(1) : (X == Y ? real(0.5) : real(0));     // share of X in it
  const real t = (a * b > real(0)) ? D : real(0);
  const real tm = real(2) * wm * t;
  const real tz = real(0.5) * (real(1) - wm) * t;
  ga = tm * wx + tz;
  gb = tm * (real(1) - wx) + tz;
}

// Reverse of vl_slope: d/da 2ab/(a+b) = 2b^2/(a+b)^2, d/db = 2a^2/(a+b)^2 where a*b > 0, else 0.
template <typename real>
__host__ __device__ __forceinline__ void vl_slope_vjp(real a, real b, real D, real& ga, real& gb) {
  ga = real(0);
  gb = real(0);
  if (!(a * b > real(0))) return;
  const real is = q_div(real(1), a + b);
  const real t = real(2) * D * is * is;
  ga = t * b * b;
  gb = t * a * a;
}

template <int LIM, typename real>
__host__ __device__ __forceinline__ void lim_slope_vjp(real a, real b, real D, real& ga, real& gb) {
  if constexpr (LIM == LIM_VL) vl_slope_vjp(a, b, D, ga, gb);
  else mc_slope_vjp(a, b, D, ga, gb);
}

// True when every component of a limited slope is zero.  The positivity fallback zeroes all
// of them; otherwise a zero component has a b <= 0 and a zero derivative, so "all zero" selects
// exactly the cells whose slope derivative vanishes as a whole.
template <typename real>
__host__ __device__ __forceinline__ bool slope_is_zero(const Prim<real>& d) {
  return d.r == real(0) && d.vx == real(0) && d.vy == real(0) && d.vz == real(0) && d.p == real(0);
}

// A_i = dL/da_i, B_i = dL/db_i of a cell (a = w_{+1} - w_0, b = w_0 - w_{-1}) from
// D = dL/d(dW_i), given whether the forward's limited slope of the cell was all zero.
template <int LIM = LIM_MC, typename real>
__host__ __device__ __forceinline__ void slope_vjp(const Prim<real>& wm, const Prim<real>& w0,
                                                   const Prim<real>& wp, bool zero, const real D[5],
                                                   real A[5], real B[5]) {
  if (zero) {
#pragma unroll
    for (int c = 0; c < 5; ++c) { A[c] = real(0); B[c] = real(0); }
    return;
  }
  lim_slope_vjp<LIM>(wp.r - w0.r, w0.r - wm.r, D[0], A[0], B[0]);
  lim_slope_vjp<LIM>(wp.vx - w0.vx, w0.vx - wm.vx, D[1], A[1], B[1]);
  lim_slope_vjp<LIM>(wp.vy - w0.vy, w0.vy - wm.vy, D[2], A[2], B[2]);
  lim_slope_vjp<LIM>(wp.vz - w0.vz, w0.vz - wm.vz, D[3], A[3], B[3]);
  lim_slope_vjp<LIM>(wp.p - w0.p, w0.p - wm.p, D[4], A[4], B[4]);
}

// Reverse of hllc() in the face frame (r, u, a, b, p) for both sides.
template <typename real>
__host__ __device__ __forceinline__ void hllc_vjp(real rL, real uL, real aL, real bL, real pL, real rR,
                                         real uR, real aR, real bR, real pR, real gamma,
                                         real gm1, real g0, real gn, real gt1, real gt2, real ge,
                                         real gL[5], real gR[5]) {
  const real cL = q_sqrt(q_div(gamma * pL, rL));
  const real cR = q_sqrt(q_div(gamma * pR, rR));
  const real xL = uL - cL, xR = uR - cR;
  const real yL = uL + cL, yR = uR + cR;
  const real SL = fmin(xL, xR);
  const real SR = fmax(yL, yR);
  const real dL = SL - uL, dR = SR - uR;
  const real num = hllc_star_num(rL, uL, pL, dL, rR, uR, pR, dR);
  const real den = hllc_star_den(rL, dL, rR, dR);
  const real Ss = q_div(num, den);
  const real iden = q_div(real(1), den);
  const bool left = (SL >= real(0)) || (Ss >= real(0));
  const bool star = !(SL >= real(0)) && (Ss >= real(0) || SR > real(0));
  const real r = left ? rL : rR, u = left ? uL : uR, a = left ? aL : aR, b = left ? bL : bR;
  const real p = left ? pL : pR, S = left ? SL : SR, d = left ? dL : dR;
  const real E = rfma(rmul(real(0.5), r), rfma(b, b, rfma(a, a, rmul(u, u))), q_div(p, gm1));
  const real mass = rmul(r, u);

  real r_ = 0, u_ = 0, a_ = 0, b_ = 0, p_ = 0, S_ = 0, Ss_ = 0, d_ = 0;
  real mass_ = g0 + gn * u + gt1 * a + gt2 * b;
  u_ += gn * mass + ge * (E + p);
  a_ += gt1 * mass;
  b_ += gt2 * mass;
  p_ += gn + ge * u;
  real E_ = ge * u;
  // reciprocals shared by the reverse sweep (quotients of the working precision, as forward)
  const real ir = q_div(real(1), r);
  if (star) {
    const real den2 = S - Ss;
    const real rd = r * d;
    const real ird = q_div(real(1), rd);
    const real iden2 = q_div(real(1), den2);
    const real coef = rd * iden2;
    const real w = p * ird;
    const real Z = Ss + w;
    const real Q = E * ir + (Ss - u) * Z;
    const real Es = coef * Q;
    S_ += g0 * (coef - r) + gn * (coef * Ss - mass) + gt1 * (coef * a - r * a) +
          gt2 * (coef * b - r * b) + ge * (Es - E);
    real coef_ = S * (g0 + gn * Ss + gt1 * a + gt2 * b);
    Ss_ += S * gn * coef;
    r_ -= S * (g0 + gt1 * a + gt2 * b);
    mass_ -= S * gn;
    a_ += S * gt1 * (coef - r);
    b_ += S * gt2 * (coef - r);
    E_ -= S * ge;
    const real Es_ = S * ge;
    coef_ += Es_ * Q;
    const real Q_ = Es_ * coef;
    E_ += Q_ * ir;
    r_ -= Q_ * E * ir * ir;
    Ss_ += Q_ * (Z + (Ss - u));
    u_ -= Q_ * Z;
    const real w_ = Q_ * (Ss - u);
    p_ += w_ * ird;
    r_ -= w_ * w * ir;        // d(p / (r d))/dr = -w / r
    d_ -= w_ * w * r * ird;   // d(p / (r d))/dd = -w / d
    r_ += coef_ * d * iden2;
    d_ += coef_ * r * iden2;
    const real dc = coef_ * coef * iden2;   // coef_ r d / den2^2
    S_ -= dc;
    Ss_ += dc;
  }
  p_ += E_ * q_div(real(1), gm1);
  r_ += E_ * real(0.5) * (u * u + a * a + b * b);
  u_ += E_ * r * u;
  a_ += E_ * r * a;
  b_ += E_ * r * b;
  r_ += mass_ * u;
  u_ += mass_ * r;
  S_ += d_;
  u_ -= d_;

  real rL_ = 0, uL_ = 0, aL_ = 0, bL_ = 0, pL_ = 0, SL_ = 0, dL_ = 0;
  real rR_ = 0, uR_ = 0, aR_ = 0, bR_ = 0, pR_ = 0, SR_ = 0, dR_ = 0;
  if (left) { rL_ = r_; uL_ = u_; aL_ = a_; bL_ = b_; pL_ = p_; SL_ = S_; }
  else      { rR_ = r_; uR_ = u_; aR_ = a_; bR_ = b_; pR_ = p_; SR_ = S_; }
  if (star) {
    const real num_ = Ss_ * iden;
    const real den_ = -num_ * Ss;
    pR_ += num_;
    pL_ -= num_;
    rL_ += num_ * uL * dL + den_ * dL;
    uL_ += num_ * rL * dL;
    dL_ += num_ * rL * uL + den_ * rL;
    rR_ -= num_ * uR * dR + den_ * dR;
    uR_ -= num_ * rR * dR;
    dR_ -= num_ * rR * uR + den_ * rR;
  }
  SL_ += dL_;
  uL_ -= dL_;
  SR_ += dR_;
  uR_ -= dR_;
  real cL_ = 0, cR_ = 0;
  if (xL < xR) { uL_ += SL_; cL_ -= SL_; }
  else if (xR < xL) { uR_ += SL_; cR_ -= SL_; }
  else { uL_ += real(0.5) * SL_; cL_ -= real(0.5) * SL_; uR_ += real(0.5) * SL_; cR_ -= real(0.5) * SL_; }
  if (yL > yR) { uL_ += SR_; cL_ += SR_; }
  else if (yR > yL) { uR_ += SR_; cR_ += SR_; }
  else { uL_ += real(0.5) * SR_; cL_ += real(0.5) * SR_; uR_ += real(0.5) * SR_; cR_ += real(0.5) * SR_; }
  // c = sqrt(gamma p / rho): dc/dp = gamma / (2 c rho), dc/drho = -c / (2 rho)
  const real hL = real(0.5) * q_div(cL_, rL), hR = real(0.5) * q_div(cR_, rR);
  pL_ += hL * q_div(gamma, cL);
  rL_ -= hL * cL;
  pR_ += hR * q_div(gamma, cR);
  rR_ -= hR * cR;
  gL[0] = rL_; gL[1] = uL_; gL[2] = aL_; gL[3] = bL_; gL[4] = pL_;
  gR[0] = rR_; gR[1] = uR_; gR[2] = aR_; gR[3] = bR_; gR[4] = pR_;
}

#if defined(__CUDA_ARCH__)
// hllc_vjp for float32 with the left and right sides in the two lanes of packed operations.  The
// forward quantities are recomputed as hllc_packed computes them (c = gamma p / sqrt(gamma p
// rho), one reciprocal for S*), so the region taken is the forward kernel's.  With
// s = 1/sqrt(gamma p rho): dc/dp = gamma s / 2 and dc/drho = -c^2 s / 2.
__device__ __forceinline__ void hllc_vjp_packed(float rL, float uL, float aL, float bL, float pL,
                                                float rR, float uR, float aR, float bR, float pR,
                                                float gamma, float gm1, float g0, float gn,
                                                float gt1, float gt2, float ge, float gL[5],
                                                float gR[5]) {
  const float2 r = f2(rL, rR), u = f2(uL, uR), pp = f2(pL, pR);
  const float2 gp = p_mul(pp, f2s(gamma));
  const float2 gpr = p_mul(gp, r);
  const float2 rs = f2(gpr.x > 0.0f ? rsqrtf(gpr.x) : 0.0f, gpr.y > 0.0f ? rsqrtf(gpr.y) : 0.0f);
  const float2 c = p_mul(gp, rs);
  const float2 um = p_sub(u, c), upc = p_add(u, c);
  const float SL = fminf(um.x, um.y), SR = fmaxf(upc.x, upc.y);
  const float2 d = p_sub(f2(SL, SR), u);
  const float2 rd = p_mul(r, d);
  const float2 t = p_sub(p_mul(rd, u), pp);
  const float Ss = q_div(t.x - t.y, rd.x - rd.y);
  const bool left = (SL >= 0.0f) || (Ss >= 0.0f);
  const bool star = !(SL >= 0.0f) && (Ss >= 0.0f || SR > 0.0f);
  const float rk = left ? rL : rR, uk = left ? uL : uR, ak = left ? aL : aR, bk = left ? bL : bR;
  const float pk = left ? pL : pR, S = left ? SL : SR, dk = left ? d.x : d.y;
  const float igm1 = 1.0f / gm1;   // uniform: hoisted out of the face loops
  const float2 ua2 = p_mul(f2(uk, ak), f2(uk, ak));
  const float q2 = ua2.x + ua2.y + bk * bk;
  const float E = pk * igm1 + 0.5f * rk * q2;
  const float mass = rk * uk;

  float mass_ = g0 + gn * uk + gt1 * ak + gt2 * bk;
  float u_ = gn * mass + ge * (E + pk);
  float2 ab_ = p_mul(f2(gt1, gt2), f2s(mass));
  float p_ = gn + ge * uk;
  float E_ = ge * uk;
  float r_ = 0.0f, S_ = 0.0f, Ss_ = 0.0f, d_ = 0.0f;
  if (star) {
    const float ir = q_div(1.0f, rk);
    const float rdk = rk * dk;
    const float ird = q_div(1.0f, rdk);
    const float iden2 = q_div(1.0f, S - Ss);
    const float coef = rdk * iden2;
    const float w = pk * ird;
    const float sdu = Ss - uk;
    const float Z = Ss + w;
    const float Q = E * ir + sdu * Z;
    const float Es = coef * Q;
    const float cr = coef - rk;
    const float G = g0 + gt1 * ak + gt2 * bk;
    S_ = G * cr + gn * (coef * Ss - mass) + ge * (Es - E);
    float coef_ = S * (G + gn * Ss);
    Ss_ = S * gn * coef;
    r_ = -S * G;
    mass_ -= S * gn;
    ab_ = p_fma(f2(gt1, gt2), f2s(S * cr), ab_);
    const float Es_ = S * ge;
    E_ -= Es_;
    coef_ += Es_ * Q;
    const float Q_ = Es_ * coef;
    E_ += Q_ * ir;
    r_ -= Q_ * E * ir * ir;
    Ss_ += Q_ * (Z + sdu);
    u_ -= Q_ * Z;
    const float w_ = Q_ * sdu;
    p_ += w_ * ird;
    r_ -= w_ * w * ir;
    d_ = -(w_ * w * rk * ird);
    r_ += coef_ * dk * iden2;
    d_ += coef_ * rk * iden2;
    const float dc = coef_ * coef * iden2;
    S_ -= dc;
    Ss_ += dc;
  }
  p_ += E_ * igm1;
  r_ += E_ * 0.5f * q2;
  const float Er = E_ * rk;
  u_ += Er * uk;
  ab_ = p_fma(f2s(Er), f2(ak, bk), ab_);
  r_ += mass_ * uk;
  u_ += mass_ * rk;
  S_ += d_;
  u_ -= d_;

  float2 rP = left ? f2(r_, 0.0f) : f2(0.0f, r_);
  float2 uP = left ? f2(u_, 0.0f) : f2(0.0f, u_);
  float2 pP = left ? f2(p_, 0.0f) : f2(0.0f, p_);
  float2 SP = left ? f2(S_, 0.0f) : f2(0.0f, S_);
  const float2 aP = left ? f2(ab_.x, 0.0f) : f2(0.0f, ab_.x);
  const float2 bP = left ? f2(ab_.y, 0.0f) : f2(0.0f, ab_.y);
  if (star) {
    // S* = num / den, num = p_R - p_L + rho_L u_L d_L - rho_R u_R d_R, den = rho_L d_L - rho_R d_R
    const float num_ = Ss_ * q_div(1.0f, rd.x - rd.y);
    const float den_ = -num_ * Ss;
    const float2 sn = f2(num_, -num_), sd = f2(den_, -den_);
    pP = p_sub(pP, sn);
    rP = p_fma(sn, p_mul(u, d), p_fma(sd, d, rP));
    uP = p_fma(sn, rd, uP);
    const float2 dP = p_fma(sn, p_mul(r, u), p_mul(sd, r));
    SP = p_add(SP, dP);
    uP = p_sub(uP, dP);
  }
  // S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R); ties split evenly
  const float wx = um.x < um.y ? 1.0f : (um.x == um.y ? 0.5f : 0.0f);
  const float wy = upc.x > upc.y ? 1.0f : (upc.x == upc.y ? 0.5f : 0.0f);
  const float2 sx = p_mul(f2(wx, 1.0f - wx), f2s(SP.x));
  const float2 sy = p_mul(f2(wy, 1.0f - wy), f2s(SP.y));
  uP = p_add(uP, p_add(sx, sy));
  const float2 c_ = p_sub(sy, sx);
  pP = p_fma(c_, p_mul(f2s(0.5f * gamma), rs), pP);
  rP = p_sub(rP, p_mul(c_, p_mul(p_mul(c, c), p_mul(rs, f2s(0.5f)))));
  gL[0] = rP.x; gL[1] = uP.x; gL[2] = aP.x; gL[3] = bP.x; gL[4] = pP.x;
  gR[0] = rP.y; gR[1] = uP.y; gR[2] = aP.y; gR[3] = bP.y; gR[4] = pP.y;
}
#endif

// HLLC VJP in the face frame: hllc_vjp_packed for the float32 device build, hllc_vjp otherwise.
template <typename real>
__host__ __device__ __forceinline__ void hllc_vjp_any(real rL, real uL, real aL, real bL, real pL,
                                                      real rR, real uR, real aR, real bR, real pR,
                                                      real gamma, real gm1, real g0, real gn,
                                                      real gt1, real gt2, real ge, real gL[5],
                                                      real gR[5]) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<real, float>::value) {
    hllc_vjp_packed(rL, uL, aL, bL, pL, rR, uR, aR, bR, pR, gamma, gm1, g0, gn, gt1, gt2, ge, gL, gR);
    return;
  }
#endif
  hllc_vjp(rL, uL, aL, bL, pL, rR, uR, aR, bR, pR, gamma, gm1, g0, gn, gt1, gt2, ge, gL, gR);
}

// Face VJP along `axis` from the reconstructed states L (upper face state of the lower cell) and
// R, and the flux gradient g[5] in (rho, m_x, m_y, m_z, E) order; returns gradients of the two
// states in (rho, v_x, v_y, v_z, P) order.
template <typename real>
__host__ __device__ __forceinline__ void face_vjp(int axis, const Prim<real>& L, const Prim<real>& R,
                                                  const real g[5], real gamma, real gm1, real gL[5],
                                                  real gR[5]) {
  real fL[5], fR[5];
  if (axis == 0) {
    hllc_vjp_any(L.r, L.vx, L.vy, L.vz, L.p, R.r, R.vx, R.vy, R.vz, R.p, gamma, gm1, g[0], g[1], g[2],
             g[3], g[4], fL, fR);
    gL[0] = fL[0]; gL[1] = fL[1]; gL[2] = fL[2]; gL[3] = fL[3]; gL[4] = fL[4];
    gR[0] = fR[0]; gR[1] = fR[1]; gR[2] = fR[2]; gR[3] = fR[3]; gR[4] = fR[4];
  } else if (axis == 1) {
    hllc_vjp_any(L.r, L.vy, L.vx, L.vz, L.p, R.r, R.vy, R.vx, R.vz, R.p, gamma, gm1, g[0], g[2], g[1],
             g[3], g[4], fL, fR);
    gL[0] = fL[0]; gL[1] = fL[2]; gL[2] = fL[1]; gL[3] = fL[3]; gL[4] = fL[4];
    gR[0] = fR[0]; gR[1] = fR[2]; gR[2] = fR[1]; gR[3] = fR[3]; gR[4] = fR[4];
  } else {
    hllc_vjp_any(L.r, L.vz, L.vx, L.vy, L.p, R.r, R.vz, R.vx, R.vy, R.p, gamma, gm1, g[0], g[3], g[1],
             g[2], g[4], fL, fR);
    gL[0] = fL[0]; gL[1] = fL[2]; gL[2] = fL[3]; gL[3] = fL[1]; gL[4] = fL[4];
    gR[0] = fR[0]; gR[1] = fR[2]; gR[2] = fR[3]; gR[3] = fR[1]; gR[4] = fR[4];
  }
}

}  // namespace dh
