// Host-side launchers of the library's kernels (implemented in hydro.cu and friends).
#pragma once
#include <cuda_runtime.h>
#include "dh_device.cuh"

namespace dh {

// Everything a stage launch needs; pointers are device pointers of the working precision.
template <typename real> struct StageArgs {
  const real* U;        // stage input: U^n (stage 1) or U1 (stage 2)
  const real* U0;       // U^n (stage 2 only)
  real* out;            // U1 (stage 1) or U^{n+1} (stage 2)
  int nx, ny, nz;
  real gamma, gm1;
  real idx, idy, idz;   // inverse cell widths
  real dx, dy, dz;      // cell widths (CFL reduction)
  StepRecord* rec;
  const double* dtp;      // time step of this stage (device scalar)
  // fused sources (stage 2 only)
  int forcing, cooling;
  const real* ahat_norm;  // 16 modes x 3 comps x (re, im), normalised
  const real* tw[3];      // per-axis twiddles: for cell i, (cos t, sin t, cos 2t, sin 2t), t = 2 pi (i+1/2)/n
  real* frow;             // scratch for the step's forcing row factors (ny nz 18 reals; the paired
                          // kernel's final stage fills and reads it, nullable otherwise)
  real t_floor, cool_frac;
  int nsub_max;
  int reduce_cfl;         // accumulate the CFL minimum of the output state
  real cool_ratio;        // > 0: also (c_cool / C) t_cool of each cell (cooling time-step limit)
  real* pre_src;          // stage 2 (nullable): also store the state before the sources
  int limiter;            // LIM_MC or LIM_VL
  // stage 3 (SSPRK3's combinations): out = w0 U0 + w1 (U + dt L(U)), (3/4, 1/4) then (1/3, 2/3);
  // final_stage: this one ends the step and takes the epilogue (pre_src, sources, finite and
  // positivity checks, CFL).  Stage 2 is RK2's final stage with weights (1/2, 1/2).
  real w0, w1;
  int final_stage;
  int count_fallbacks;    // add the own cells' positivity fallbacks to rec->slope_fallbacks
};

// stage 1: U + dt L(U); 2: RK2's final stage; 3: the weighted combination of SSPRK3.
// `launched` (nullable) receives the number of kernels enqueued.
template <typename real>
cudaError_t launch_stage(int stage, const StageArgs<real>& a, cudaStream_t s, int* launched = nullptr);
// The same stage by the paired kernel (hydro_pair.cu) when the grid has whole 64 x 8 tiles and
// the state takes tensor-map copies: returns false (nothing launched) otherwise; err is the
// launches' status and launched their number (the final stage with forcing first fills the
// forcing row-factor table).
template <typename real>
bool launch_stage_pair(int stage, const StageArgs<real>& a, cudaStream_t s, cudaError_t& err, int& launched);

struct BeginArgs {
  StepRecord* rec;
  double dt_fixed, cfl, dt_max;
  int precision;            // 0 float, 1 double
  int forcing;
  double* ahat;             // 96 doubles (re, im) — unnormalised OU state
  double* ahat_prev;        // copy before this step's update
  void* ahat_norm;          // 96 reals of the working precision
  unsigned long long seed;
  double tau, arms;
  int hold;                 // keep the table (no draw, no update), only renormalise it
  // projected draws made ahead (launch_ou_draws) for steps [draw_first, draw_first +
  // draw_count): 96 doubles per step; a step outside the range draws in the kernel
  const double* draws;
  long long draw_first;
  int draw_count;
};
cudaError_t launch_step_begin(const BeginArgs& a, cudaStream_t s);
// The projected OU draws of steps first .. first + count - 1 (one CTA per step) into out.
constexpr int OU_DRAW_BATCH = 128;
cudaError_t launch_ou_draws(unsigned long long seed, long long first, int count, double* out,
                            cudaStream_t s);
cudaError_t launch_forcing_init(double* ahat, unsigned long long seed, cudaStream_t s);

template <typename real>
cudaError_t launch_cfl_reduce(const real* U, int nx, int ny, int nz, real gamma, real dx, real dy,
                              real dz, real cool_ratio, real t_floor, StepRecord* rec,
                              cudaStream_t s);

template <typename real>
cudaError_t launch_totals(const real* U, long long n3, double* partials, int nblocks,
                          double* out5, cudaStream_t s);

template <typename real>
cudaError_t launch_forcing_field(const real* ahat_norm, const real* const tw[3], int nx, int ny,
                                 int nz, real* a_out, cudaStream_t s);

// minima over cells of rho and P into out2 (device); partials holds 2 * nblocks doubles
template <typename real>
cudaError_t launch_minima(const real* U, long long n3, double gamma, double* partials, int nblocks,
                          double* out2, cudaStream_t s);

int totals_blocks();
// Streaming multiprocessors of the current device.
int sm_count();
// Planes per z chunk for a kernel whose CTAs each march one column tile through a chunk of
// planes: the tiles x chunks CTAs run in waves of sm_count() x resident_per_sm, and the choice
// maximises the filled fraction of the waves times zc / (zc + prologue), where `prologue` is the
// cost of a chunk's start in planes.  Chunks hold at least `min_planes` planes (all nz if nz <
// 2 min_planes).
int wave_zchunk(long long tiles, int nz, int resident_per_sm, double prologue, int min_planes = 8);

// Adjoint of one RK2 stage (adjoint.cu):
//   lam_in = c1 * lam_out + c2 * extra + (dL/dU)^T (beta * dt * lam_out),  L the unsplit RHS at U.
template <typename real> struct AdjointArgs {
  const real* U;         // stage input state
  const real* lam_out;   // gradient with respect to the stage output
  const real* extra;     // added with weight c2 (nullable)
  real* lam_in;          // result
  int nx, ny, nz;
  real gamma, gm1, idx, idy, idz;
  real c1, c2, beta;
  const double* dtp;
  const real* extra2;    // added with weight c3 (nullable; SSPRK3's first stage)
  real c3;
  int limiter;           // LIM_MC or LIM_VL
  unsigned* flags;       // step record flags: FLAG_TIMEOUT if a bounded copy wait gives up
};
// Adjoint of the operator-split sources of one step (forcing kick, gravity kick, cooling),
// pointwise: lamH = (dF/dU)^T (dG/dU)^T (dC/dU)^T lam at the state UH the sources were applied
// to, and with gravity h = dL/dg (the potential's part is added by a Poisson solve).
template <typename real> struct SourceAdjArgs {
  const real* lam;        // lambda of the state after the sources
  const real* UH;         // state after the RK2 step, before the sources
  real* lamH;             // lambda of UH
  const real* tab;        // normalised OU table of the step (nullable: no forcing)
  const real* tw[3];      // forcing twiddles
  int nx, ny, nz;
  int cooling;
  real gm1, t_floor, cool_frac;
  int nsub_max;
  const double* dtp;
  const float* phi;       // potential of the step, float-float planar (nullable: no gravity)
  double* h;              // gravity: dL/dg, 3 planes (output)
  double i2h;             // 1 / (2 dx)
};
template <typename real>
cudaError_t launch_source_adjoint(const SourceAdjArgs<real>& a, cudaStream_t s);

template <typename real>
cudaError_t launch_stage_adjoint(const AdjointArgs<real>& a, cudaStream_t s);

}  // namespace dh
