// Source terms and the CFL time of two cells at once (lanes x and y of pair_t, as in
// dh_pair.cuh), each lane with the roundings of the scalar function it pairs, so a cell's result
// does not depend on its lane and equals the scalar function's bit for bit.  Used by the paired
// stage kernel (hydro_pair.cu) and the paired gravity-source kernel (multigrid.cu).
#pragma once
#include <math.h>

#include <type_traits>

#include "dh_pair.cuh"
#include "dh_sources.cuh"

namespace dh {

// Cooling of two cells (Sec. 4.3): cooling_energy's arithmetic on both lanes at once, with the
// same roundings, so each lane gets that function's result bit for bit.  The trapezoid step
// (one substep) runs packed; a pair with a subcycled lane takes the scalar function per lane.
// Lanes at or below the floor energy keep E (their packed values, possibly not finite, are
// discarded).
template <typename real>
__device__ __forceinline__ pair_t<real> cooling_energy2(pair_t<real> r, pair_t<real> mx, pair_t<real> my,
                                                        pair_t<real> mz, pair_t<real> E, real dt, real gm1,
                                                        real T_floor, real frac, int nsub_max,
                                                        unsigned& flags, int& nsub_seen) {
  using P = pair_t<real>;
  const P ir = pdiv(pset(real(1)), r);
  const P kin = pmul(pmul(pset(real(0.5)), pfma(mz, mz, pfma(my, my, pmul(mx, mx)))), ir);
  const P Eth = psub(E, kin);
  const P Efl = pmul(pmul(r, pset(T_floor)), pset(real(1) / gm1));
  const bool ca = Eth.x > Efl.x, cb = Eth.y > Efl.y;
  if (!ca && !cb) return E;
  const P r2 = pmul(r, r);
  auto rate = [&](P e) {
    const P q = pmul(pmul(pset(gm1), e), ir);
    return pneg(pmul(r2, pmk(q_sqrt(q.x), q_sqrt(q.y))));
  };
  const P Ed0 = rate(Eth);
  const P raw = pdiv(pmul(pset(dt), pneg(Ed0)), pmul(pset(frac), Eth));
  // a lane takes the packed trapezoid when its substep count ceil(raw) is 1
  const bool one_a = !ca || ceil(raw.x) == real(1), one_b = !cb || ceil(raw.y) == real(1);
  if (!(one_a && one_b)) {
    const real ea = ca ? cooling_energy(r.x, mx.x, my.x, mz.x, E.x, dt, gm1, T_floor, frac, nsub_max,
                                        flags, nsub_seen) : E.x;
    const real eb = cb ? cooling_energy(r.y, mx.y, my.y, mz.y, E.y, dt, gm1, T_floor, frac, nsub_max,
                                        flags, nsub_seen) : E.y;
    return pmk(ea, eb);
  }
  const P Ep = pmax(Efl, pfma(pset(dt), Ed0, Eth));
  const P Ed1 = rate(Ep);
  const P Edp = pmk(Ep.x > Efl.x ? Ed1.x : real(0), Ep.y > Efl.y ? Ed1.y : real(0));
  const P En = padd(kin, pmax(Efl, pfma(pset(real(0.5) * dt), padd(Ed0, Edp), Eth)));
  return pmk(ca ? En.x : E.x, cb ? En.y : E.y);
}

// CFL time min_a dx_a / (|v_a| + c) of two cells (App. A.4) with cfl_time's arithmetic on both
// lanes: the primitive recovery and the sound speed of the working precision, the same
// operations in the same order, each lane rounded once, so each lane has cfl_time's bits (the
// step's CFL minimum then equals that of cfl_reduce_kernel on the same state).  The pressure is
// returned for the positivity check.
template <typename real>
__device__ __forceinline__ pair_t<real> cfl_time2(const pair_t<real> u[5], real gamma, real gm1, real dx,
                                                  real dy, real dz, pair_t<real>& pres) {
  using P = pair_t<real>;
  P vx, vy, vz, v2;
  if constexpr (std::is_same<real, float>::value) {
    const P ir = pdiv(pset(1.0f), u[0]);
    vx = pmul(u[1], ir); vy = pmul(u[2], ir); vz = pmul(u[3], ir);
    v2 = pfma(vz, vz, padd(pmul(vx, vx), pmul(vy, vy)));
  } else {
    vx = pdiv(u[1], u[0]); vy = pdiv(u[2], u[0]); vz = pdiv(u[3], u[0]);
    v2 = pfma(vz, vz, pfma(vy, vy, pmul(vx, vx)));
  }
  pres = pmul(pset(gm1), pfma(pmul(pset(real(-0.5)), u[0]), v2, u[4]));
  P c;
  const P gp = pmul(pset(gamma), pres);
  if constexpr (std::is_same<real, float>::value) {
    const P gpr = pmul(gp, u[0]);
    c = pmul(gp, pmk(gpr.x > 0.0f ? rsqrtf(gpr.x) : 0.0f, gpr.y > 0.0f ? rsqrtf(gpr.y) : 0.0f));
    c = pmk(gpr.x > 0.0f ? c.x : 0.0f, gpr.y > 0.0f ? c.y : 0.0f);
  } else {
    const P q = pdiv(gp, u[0]);
    c = pmk(sqrt(q.x), sqrt(q.y));
  }
  const P tx = pdiv(pset(dx), padd(pmk(fabs(vx.x), fabs(vx.y)), c));
  const P ty = pdiv(pset(dy), padd(pmk(fabs(vy.x), fabs(vy.y)), c));
  const P tz = pdiv(pset(dz), padd(pmk(fabs(vz.x), fabs(vz.y)), c));
  return pmin(pmin(tx, ty), tz);
}

}  // namespace dh
