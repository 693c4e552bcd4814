// Context layout and internal hooks shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dh.h"
#include "dh_kernels.h"

struct dh_ctx {
  dh_config cfg;
  int prec = DH_F32;
  cudaStream_t stream = nullptr;
  long long n3 = 0;
  size_t state_bytes = 0;
  void* U[2] = {nullptr, nullptr};   // ping-pong state buffers
  int cur = 0;                       // index of the current state
  void* U1 = nullptr;                // RK2 intermediate stage
  dh::StepRecord* rec = nullptr;     // device step record
  dh::StepRecord host_rec{};         // host copy after the last synchronisation
  int pending_steps = 0;             // steps enqueued since the last synchronisation
  double* ahat = nullptr;            // OU mode table (96 doubles), unnormalised
  double* ahat_prev = nullptr;       // table before the last update (rollback)
  void* ahat_norm = nullptr;         // normalised table in the working precision
  void* frow = nullptr;              // forcing row factors of the step (ny nz 18 reals)
  void* tw[3] = {nullptr, nullptr, nullptr};  // per-axis forcing twiddles
  int ou_hold = 0;                   // 1: steps keep the forcing table as set (no OU update)
  double* ou_draws = nullptr;        // projected draws of steps [ou_draw_first, + ou_draw_count)
  long long ou_draw_first = 0;
  int ou_draw_count = 0;
  double* partials = nullptr;        // totals: per-block partial sums
  double* totals = nullptr;          // totals: 5 doubles
  bool initialized = false;
  std::string err;
  // profiling
  bool prof_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  std::vector<int> prof_kinds;
  double prof_ms[DH_KERNEL_KINDS] = {0};
  long long prof_count[DH_KERNEL_KINDS] = {0};
  long long launches = 0;
  // multigrid (gravity)
  struct MG* mg = nullptr;
  // adjoint work space
  struct AdjointSpace* adj = nullptr;
  // corrector network (dh_set_corrector)
  struct dh_cnn* cnn = nullptr;
  bool correct_each_step = false;    // dh_set_correct_every_step: the step applies the corrector
};

namespace dh {
// cnn.cu: enqueues the corrector on U (float32, in place) inside a step: no synchronisation;
// after a fatal flag it changes nothing, and a non-finite result fails the step
cudaError_t correct_in_step(dh_ctx* c, float* U);

void prof_begin(dh_ctx* c, int kind);
void prof_end(dh_ctx* c, int launches);
void prof_fold(dh_ctx* c);

// multigrid.cu
std::string mg_validate(const dh_config& c);
cudaError_t mg_allocate(dh_ctx* c);
void mg_setup_host(dh_ctx* c);
cudaError_t mg_reset(dh_ctx* c);
void mg_last(const dh_ctx* c, int* cycles, double* rel_residual);   // the last solve's outcome
void mg_free(dh_ctx* c);
void* mg_phi(dh_ctx* c);   // the potential, float-float planar, 8 B per cell (warm start of the next solve)
// Poisson solve on the density of Ustar, then forcing -> gravity -> cooling in place.  tab:
// normalised OU table (null: the context's current one); dtp: the step's dt on the device;
// in_step: a step of the context (records flags and the CFL minimum) rather than a replay.
template <typename real>
cudaError_t gravity_sources(dh_ctx* c, void* Ustar, const void* tab, const double* dtp,
                            bool in_step);
// A x = rhs - <rhs> by V-cycles (x: warm start and result, <x> = 0), for the adjoint.
cudaError_t mg_solve_rhs(dh_ctx* c, const double* rhs, float* x);   // x float-float planar

// adjoint.cu
void adjoint_free(dh_ctx* c);
}  // namespace dh

// dh_api.cu: step machinery shared with the adjoint driver
// Optional extra outputs of one step (each nullable): the stage-1 state, SSPRK3's second-stage
// state and, with fused sources, the state before the sources.  The adjoint's forward sweep
// keeps its last segment this way instead of replaying it.
struct StepCapture {
  void* u1 = nullptr;
  void* u2 = nullptr;
  void* pre_src = nullptr;
};
cudaError_t dh_enqueue_step_f32(dh_ctx* c, double dt_fixed,    // dt_fixed <= 0: CFL
                                const StepCapture* cap = nullptr);
cudaError_t dh_enqueue_step_f64(dh_ctx* c, double dt_fixed, const StepCapture* cap = nullptr);
dh_status dh_finish_steps(dh_ctx* c);
// message returned by dh_last_error(NULL)
void dh_set_global_error(const std::string& msg);
// recompute the CFL minimum of the current state (after an external change of the state)
dh_status dh_refresh_cfl(dh_ctx* c);
extern "C" void dh_cnn_destroy(struct dh_cnn* c);
