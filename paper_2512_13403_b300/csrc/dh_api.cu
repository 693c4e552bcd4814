// C ABI of the library (declared in include/dh.h): context life cycle, state transfer and the
// host-side orchestration of one step — prologue (dt, OU update), RK2 stage 1, RK2 stage 2 with
// the fused sources and the CFL reduction — all on the context's stream with no host
// synchronisation inside dh_advance.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dh.h"
#include "dh_internal.h"

using namespace dh;

static thread_local std::string g_create_error;

void dh_set_global_error(const std::string& msg) { g_create_error = msg; }

static dh_status fail(dh_ctx* c, dh_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

static dh_status cuda_fail(dh_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, DH_ERR_CUDA, m);
}

#define DH_CUDA(c, call)                                   \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, #call); \
  } while (0)

extern "C" void dh_config_default(dh_config* cfg, int nx, int ny, int nz) {
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->nx = nx; cfg->ny = ny; cfg->nz = nz;
  cfg->precision = DH_F32;
  cfg->dx = nx > 0 ? 1.0 / nx : 0.0;
  cfg->dy = ny > 0 ? 1.0 / ny : 0.0;
  cfg->dz = nz > 0 ? 1.0 / nz : 0.0;
  cfg->gamma = 5.0 / 3.0;
  cfg->cfl = 0.4;
  cfg->dt_max = INFINITY;
  cfg->forcing = 0; cfg->ou_tau = 0.5; cfg->ou_arms = 1.0; cfg->ou_seed = 1;
  cfg->cooling = 0; cfg->t_floor = 0.05; cfg->cool_frac = 0.1; cfg->nsub_max = 1024;
  cfg->gravity = 0; cfg->four_pi_G = 1.0; cfg->mg_tol = 1e-6; cfg->mg_max_cycles = 30;
  cfg->mg_pre = 2; cfg->mg_post = 2;
  cfg->mg_smoother = 0; cfg->mg_omega = 2.0 / 3.0; cfg->mg_cycle = 1;
  cfg->limiter = 0; cfg->integrator = 2;
  cfg->c_cool = INFINITY;
}

static std::string validate(const dh_config& c) {
  if (c.nx < 4 || c.ny < 4 || c.nz < 4) return "every grid dimension must be >= 4";
  if ((long long)c.nx * c.ny * c.nz > (1LL << 31)) return "grid larger than 2^31 cells";
  if (c.precision != DH_F32 && c.precision != DH_F64) return "precision must be DH_F32 or DH_F64";
  if (!(c.dx > 0 && c.dy > 0 && c.dz > 0)) return "cell widths must be positive";
  if (!(c.gamma > 1.0)) return "gamma must exceed 1";
  if (!(c.cfl > 0.0)) return "cfl must be positive";
  if (!(c.dt_max > 0.0)) return "dt_max must be positive";
  if (c.limiter != 0 && c.limiter != 1) return "limiter must be 0 (MC) or 1 (van Leer)";
  if (c.integrator != 2 && c.integrator != 3) return "integrator must be 2 (RK2) or 3 (SSPRK3)";
  if (!(c.c_cool > 0.0)) return "c_cool must be positive (+inf: no cooling time-step limit)";
  if (c.forcing) {
    if (c.nx < 5 || c.ny < 5 || c.nz < 5) return "forcing needs every dimension >= 5";
    if (!(c.ou_tau > 0.0) || !(c.ou_arms >= 0.0)) return "ou_tau must be > 0 and ou_arms >= 0";
  }
  if (c.cooling) {
    if (!(c.t_floor >= 0.0)) return "t_floor must be >= 0";
    if (!(c.cool_frac > 0.0)) return "cool_frac must be > 0";
    if (c.nsub_max < 1) return "nsub_max must be >= 1";
  }
  if (c.gravity) {
    std::string m = mg_validate(c);
    if (!m.empty()) return m;
  }
  return "";
}

static size_t esize(const dh_ctx* c) { return c->prec == DH_F64 ? 8 : 4; }

template <typename real>
static void upload_twiddles(dh_ctx* c) {
  const int n[3] = {c->cfg.nx, c->cfg.ny, c->cfg.nz};
  for (int a = 0; a < 3; ++a) {
    std::vector<real> t(4 * (size_t)n[a]);
    for (int i = 0; i < n[a]; ++i) {
      // cell centre x~ = (i + 1/2) / n: exp(2 pi i q x~) for q = 1, 2
      const double th = 2.0 * M_PI * (i + 0.5) / n[a];
      t[4 * i + 0] = (real)std::cos(th);
      t[4 * i + 1] = (real)std::sin(th);
      t[4 * i + 2] = (real)std::cos(2.0 * th);
      t[4 * i + 3] = (real)std::sin(2.0 * th);
    }
    cudaMemcpy(c->tw[a], t.data(), t.size() * sizeof(real), cudaMemcpyHostToDevice);
  }
}

extern "C" dh_status dh_create(const dh_config* cfg, void* stream, dh_ctx** out) {
  if (!cfg || !out) return fail(nullptr, DH_ERR_ARG, "null argument");
  *out = nullptr;
  std::string msg = validate(*cfg);
  if (!msg.empty()) return fail(nullptr, DH_ERR_ARG, msg);
  dh_ctx* c = new dh_ctx();
  c->cfg = *cfg;
  c->prec = cfg->precision;
  c->stream = (cudaStream_t)stream;
  c->n3 = (long long)cfg->nx * cfg->ny * cfg->nz;
  c->state_bytes = (size_t)c->n3 * 5 * esize(c);
  auto alloc = [&](void** p, size_t bytes) -> cudaError_t { return cudaMalloc(p, bytes); };
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = alloc(&c->U[b], c->state_bytes);
  if (e == cudaSuccess) e = alloc(&c->U1, c->state_bytes);
  if (e == cudaSuccess) e = alloc((void**)&c->rec, sizeof(StepRecord));
  if (e == cudaSuccess) e = alloc((void**)&c->ahat, 96 * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->ahat_prev, 96 * sizeof(double));
  if (e == cudaSuccess) e = alloc(&c->ahat_norm, 96 * esize(c));
  if (e == cudaSuccess && cfg->forcing) e = alloc((void**)&c->ou_draws, OU_DRAW_BATCH * 96 * sizeof(double));
  if (e == cudaSuccess && cfg->forcing)
    e = alloc(&c->frow, (size_t)cfg->ny * cfg->nz * 18 * esize(c));
  if (e == cudaSuccess) e = alloc((void**)&c->partials, (size_t)totals_blocks() * 5 * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->totals, 5 * sizeof(double));
  const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = alloc(&c->tw[a], 4 * (size_t)n[a] * esize(c));
  if (e == cudaSuccess && cfg->gravity) e = mg_allocate(c);
  if (e != cudaSuccess) {
    std::string m = std::string("device allocation failed: ") + cudaGetErrorString(e);
    dh_destroy(c);
    cudaGetLastError();
    return fail(nullptr, DH_ERR_CUDA, m);
  }
  if (c->prec == DH_F64) upload_twiddles<double>(c); else upload_twiddles<float>(c);
  {
    // a defined step record from the start: no flags, no failure, CFL minimum +inf
    StepRecord r;
    std::memset(&r, 0, sizeof(r));
    r.fail_step = -1;
    r.cfl_min_bits = c->prec == DH_F32 ? (unsigned long long)0x7f800000u : 0x7ff0000000000000ull;
    c->host_rec = r;
    cudaMemcpy(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice);
  }
  if (cfg->gravity) mg_setup_host(c);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::string m = std::string("setup failed: ") + cudaGetErrorString(e);
    dh_destroy(c);
    return fail(nullptr, DH_ERR_CUDA, m);
  }
  *out = c;
  return DH_OK;
}

extern "C" void dh_destroy(dh_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  for (int b = 0; b < 2; ++b) cudaFree(c->U[b]);
  cudaFree(c->U1);
  cudaFree(c->rec);
  cudaFree(c->ahat);
  cudaFree(c->ahat_prev);
  cudaFree(c->ou_draws);
  cudaFree(c->ahat_norm);
  cudaFree(c->frow);
  cudaFree(c->partials);
  cudaFree(c->totals);
  for (int a = 0; a < 3; ++a) cudaFree(c->tw[a]);
  mg_free(c);
  adjoint_free(c);
  if (c->cnn) dh_cnn_destroy(c->cnn);
  for (auto& ev : c->prof_events) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  delete c;
}

// ---------------------------------------------------------------------------------------------
// Launch bookkeeping: counts every kernel launch and, when profiling, brackets it with events.
void dh::prof_begin(dh_ctx* c, int kind) {
  if (!c->prof_on) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, c->stream);
  c->prof_events.push_back({a, b});
  c->prof_kinds.push_back(kind);
}

void dh::prof_end(dh_ctx* c, int launches) {
  c->launches += launches;
  if (!c->prof_on) return;
  cudaEventRecord(c->prof_events.back().second, c->stream);
  if (c->prof_events.size() >= 4096) prof_fold(c);
}

void dh::prof_fold(dh_ctx* c) {
  if (c->prof_events.empty()) return;
  cudaEventSynchronize(c->prof_events.back().second);
  for (size_t i = 0; i < c->prof_events.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->prof_events[i].first, c->prof_events[i].second);
    const int k = c->prof_kinds[i];
    c->prof_ms[k] += ms;
    c->prof_count[k] += 1;
    cudaEventDestroy(c->prof_events[i].first);
    cudaEventDestroy(c->prof_events[i].second);
  }
  c->prof_events.clear();
  c->prof_kinds.clear();
}

// ---------------------------------------------------------------------------------------------
// c_cool / C: the reductions take min over cells of min(CFL time, (c_cool / C) t_cool), so that
// C times the minimum is min(CFL step, c_cool min t_cool); 0 when the limit is off.
template <typename real>
static real cool_ratio(const dh_config& g) {
  return g.cooling && std::isfinite(g.c_cool) ? (real)(g.c_cool / g.cfl) : real(0);
}

template <typename real>
static cudaError_t cfl_reduce_current(dh_ctx* c) {
  const dh_config& g = c->cfg;
  prof_begin(c, DH_KERNEL_REDUCE);
  cudaError_t e = launch_cfl_reduce<real>((const real*)c->U[c->cur], g.nx, g.ny, g.nz,
                                          (real)g.gamma, (real)g.dx, (real)g.dy, (real)g.dz,
                                          cool_ratio<real>(g), (real)g.t_floor, c->rec, c->stream);
  prof_end(c, 1);
  return e;
}

__global__ void set_u64_kernel(unsigned long long* p, unsigned long long v) { *p = v; }

static cudaError_t reset_cfl_bits(dh_ctx* c) {
  const unsigned long long inf_bits =
      c->prec == DH_F32 ? (unsigned long long)0x7f800000u : 0x7ff0000000000000ull;
  return cudaMemcpyAsync(&c->rec->cfl_min_bits, &inf_bits, sizeof(inf_bits),
                         cudaMemcpyHostToDevice, c->stream);
}

extern "C" dh_status dh_init_state(dh_ctx* c, const void* U, int on_device) {
  if (!c || !U) return fail(c, DH_ERR_ARG, "null argument");
  DH_CUDA(c, cudaMemcpyAsync(c->U[0], U, c->state_bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
  c->cur = 0;
  c->pending_steps = 0;
  StepRecord r;
  std::memset(&r, 0, sizeof(r));
  r.fail_step = -1;
  r.cfl_min_bits = c->prec == DH_F32 ? (unsigned long long)0x7f800000u : 0x7ff0000000000000ull;
  c->host_rec = r;
  DH_CUDA(c, cudaMemcpyAsync(c->rec, &c->host_rec, sizeof(r), cudaMemcpyHostToDevice, c->stream));
  if (c->cfg.forcing) {
    prof_begin(c, DH_KERNEL_PROLOGUE);
    DH_CUDA(c, launch_forcing_init(c->ahat, c->cfg.ou_seed, c->stream));
    prof_end(c, 1);
  }
  if (c->cfg.gravity) DH_CUDA(c, mg_reset(c));
  DH_CUDA(c, c->prec == DH_F64 ? cfl_reduce_current<double>(c) : cfl_reduce_current<float>(c));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  c->initialized = true;
  return DH_OK;
}

static dh_status finish_steps(dh_ctx* c, long long nstep_before);

extern "C" dh_status dh_get_state(dh_ctx* c, void* U, int on_device) {
  if (!c || !U) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  // settle enqueued steps first: after a failed one the current state is the last good step
  const dh_status st = c->pending_steps > 0 ? finish_steps(c, c->host_rec.nstep - c->pending_steps) : DH_OK;
  DH_CUDA(c, cudaMemcpyAsync(U, c->U[c->cur], c->state_bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

template <typename real>
static StageArgs<real> stage_args(dh_ctx* c) {
  const dh_config& g = c->cfg;
  StageArgs<real> a;
  std::memset(&a, 0, sizeof(a));
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.gamma = (real)g.gamma; a.gm1 = (real)(g.gamma - 1.0);
  a.idx = (real)(1.0 / g.dx); a.idy = (real)(1.0 / g.dy); a.idz = (real)(1.0 / g.dz);
  a.dx = (real)g.dx; a.dy = (real)g.dy; a.dz = (real)g.dz;
  a.rec = c->rec;
  a.dtp = &c->rec->dt;
  a.ahat_norm = (const real*)c->ahat_norm;
  for (int q = 0; q < 3; ++q) a.tw[q] = (const real*)c->tw[q];
  a.frow = (real*)c->frow;
  a.t_floor = (real)g.t_floor; a.cool_frac = (real)g.cool_frac; a.nsub_max = g.nsub_max;
  a.cool_ratio = cool_ratio<real>(g);
  a.limiter = g.limiter;
  a.w0 = real(0.5); a.w1 = real(0.5);
  a.final_stage = 1;
  a.count_fallbacks = 1;
  return a;
}

// Enqueues one full step reading U[cur] and writing U[1-cur]; no synchronisation.
template <typename real>
static cudaError_t enqueue_step(dh_ctx* c, double dt_fixed, const StepCapture* cap) {
  const dh_config& g = c->cfg;
  BeginArgs b;
  b.rec = c->rec; b.dt_fixed = dt_fixed; b.cfl = g.cfl; b.dt_max = g.dt_max;
  b.precision = c->prec == DH_F64 ? 1 : 0;
  b.forcing = g.forcing; b.ahat = c->ahat; b.ahat_prev = c->ahat_prev; b.ahat_norm = c->ahat_norm;
  b.seed = g.ou_seed; b.tau = g.ou_tau; b.arms = g.ou_arms;
  b.hold = c->ou_hold;
  b.draws = nullptr;
  b.draw_first = 0;
  b.draw_count = 0;
  cudaError_t e = cudaSuccess;
  if (g.forcing && !c->ou_hold && c->ou_draws) {
    // the draw this step takes if every enqueued step succeeds (otherwise the kernel sees a
    // different step count and draws itself); refill the table when it is not covered
    const long long d = c->host_rec.nstep + c->pending_steps + 1;
    if (c->ou_draw_count == 0 || d < c->ou_draw_first || d >= c->ou_draw_first + c->ou_draw_count) {
      prof_begin(c, DH_KERNEL_PROLOGUE);
      e = launch_ou_draws(g.ou_seed, d, OU_DRAW_BATCH, c->ou_draws, c->stream);
      prof_end(c, 1);
      if (e != cudaSuccess) return e;
      c->ou_draw_first = d;
      c->ou_draw_count = OU_DRAW_BATCH;
    }
    b.draws = c->ou_draws;
    b.draw_first = c->ou_draw_first;
    b.draw_count = c->ou_draw_count;
  }
  prof_begin(c, DH_KERNEL_PROLOGUE);
  e = launch_step_begin(b, c->stream);
  prof_end(c, 1);
  if (e != cudaSuccess) return e;

  StageArgs<real> a = stage_args<real>(c);
  const real* Un = (const real*)c->U[c->cur];
  real* Unew = (real*)c->U[1 - c->cur];
  const bool rk3 = g.integrator == 3;
  // RK2: U^n -> U1 (scratch) -> U^{n+1}.  SSPRK3: U^n -> U1 (in the output buffer) -> U2
  // (scratch) -> U^{n+1}; U^n is never written, so it stays the last good state.
  real* Ust1 = cap && cap->u1 ? (real*)cap->u1 : (rk3 ? Unew : (real*)c->U1);
  a.U = Un; a.U0 = nullptr; a.out = Ust1;
  int nl = 1;
  prof_begin(c, DH_KERNEL_STAGE1);
  e = launch_stage<real>(1, a, c->stream, &nl);
  prof_end(c, nl);
  if (e != cudaSuccess) return e;
  const real* Ulast = Ust1;
  if (rk3) {
    StageArgs<real> m = a;
    m.U = Ust1; m.U0 = Un; m.out = cap && cap->u2 ? (real*)cap->u2 : (real*)c->U1;
    m.w0 = real(0.75); m.w1 = real(0.25);
    m.final_stage = 0;
    prof_begin(c, DH_KERNEL_STAGE1);
    e = launch_stage<real>(3, m, c->stream, &nl);
    prof_end(c, nl);
    if (e != cudaSuccess) return e;
    Ulast = m.out;
    a.w0 = real(1.0 / 3.0); a.w1 = real(2.0 / 3.0);
  }

  a.U = Ulast; a.U0 = Un; a.out = Unew;
  const bool fuse = !g.gravity;
  // with the corrector in the step, the next step's CFL minimum is the corrected state's
  const bool correct = c->correct_each_step && std::is_same<real, float>::value;
  a.forcing = fuse ? g.forcing : 0;
  a.cooling = fuse ? g.cooling : 0;
  a.reduce_cfl = fuse && !correct ? 1 : 0;
  a.pre_src = fuse && cap ? (real*)cap->pre_src : nullptr;
  prof_begin(c, DH_KERNEL_STAGE2);
  e = launch_stage<real>(rk3 ? 3 : 2, a, c->stream, &nl);
  prof_end(c, nl);
  if (e != cudaSuccess) return e;
  if (!fuse) {
    e = gravity_sources<real>(c, Unew, nullptr, &c->rec->dt, true);
    if (e != cudaSuccess) return e;
  }
  if (correct) {
    // Sec. 7: the corrector after the coarse step, in place on the new state, then the CFL
    // minimum of the corrected state (the sources' reduction, if any, is discarded)
    prof_begin(c, DH_KERNEL_CONV);
    e = correct_in_step(c, (float*)Unew);
    prof_end(c, 0);
    if (e != cudaSuccess) return e;
    set_u64_kernel<<<1, 1, 0, c->stream>>>(&c->rec->cfl_min_bits, (unsigned long long)0x7f800000u);
    prof_begin(c, DH_KERNEL_REDUCE);
    e = launch_cfl_reduce<real>((const real*)Unew, g.nx, g.ny, g.nz, (real)g.gamma, (real)g.dx,
                                (real)g.dy, (real)g.dz, cool_ratio<real>(g), (real)g.t_floor,
                                c->rec, c->stream);
    prof_end(c, 2);
    if (e != cudaSuccess) return e;
  }
  c->cur = 1 - c->cur;
  c->pending_steps += 1;
  return cudaSuccess;
}

// Reads the device record after a batch of steps; on a fatal flag rolls the host view back to
// the last good step (whose state is the input buffer of the failing step).
static dh_status finish_steps(dh_ctx* c, long long nstep_before) {
  DH_CUDA(c, cudaMemcpyAsync(&c->host_rec, c->rec, sizeof(StepRecord), cudaMemcpyDeviceToHost,
                             c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  const int pending = c->pending_steps;
  c->pending_steps = 0;
  StepRecord& r = c->host_rec;
  if (r.flags & FATAL_FLAGS) {
    // r.nstep counts the failing step (its prologue ran); later steps were skipped.
    const long long failed = r.fail_step;
    const long long done_ok = failed - nstep_before;  // good steps in this batch
    // buffer parity: after `pending` swaps cur points at the output of the last enqueued step
    const int cur_before = (int)((c->cur + pending) & 1);
    c->cur = (int)((cur_before + done_ok) & 1);
    r.t -= r.dt;
    r.nstep = failed;
    unsigned fl = r.flags;
    r.flags = 0;
    r.fail_step = -1;
    cudaMemcpyAsync(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice, c->stream);
    if (c->cfg.forcing)
      cudaMemcpyAsync(c->ahat, c->ahat_prev, 96 * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->stream);
    // the failing stage may have stopped part-way: recompute the CFL minimum of the restored state
    reset_cfl_bits(c);
    if (c->prec == DH_F64) cfl_reduce_current<double>(c); else cfl_reduce_current<float>(c);
    cudaStreamSynchronize(c->stream);
    if (fl & FLAG_TIMEOUT)
      return fail(c, DH_ERR_CUDA, "a kernel's bounded wait for its own copies gave up in step " +
                                      std::to_string(failed));
    if (fl & FLAG_MG_NOCONV)
      return fail(c, DH_ERR_MG_NOCONV, "multigrid did not converge in step " + std::to_string(failed));
    if (fl & FLAG_NONFINITE)
      return fail(c, DH_ERR_NONFINITE, "non-finite state in step " + std::to_string(failed));
    return fail(c, DH_ERR_POSITIVITY, "rho or P not positive after step " + std::to_string(failed));
  }
  return DH_OK;
}

dh_status dh_refresh_cfl(dh_ctx* c) {
  // stream-ordered: the next step reads the minimum on the device
  DH_CUDA(c, reset_cfl_bits(c));
  DH_CUDA(c, c->prec == DH_F64 ? cfl_reduce_current<double>(c) : cfl_reduce_current<float>(c));
  return DH_OK;
}

cudaError_t dh_enqueue_step_f32(dh_ctx* c, double dt, const StepCapture* cap) {
  return enqueue_step<float>(c, dt, cap);
}
cudaError_t dh_enqueue_step_f64(dh_ctx* c, double dt, const StepCapture* cap) {
  return enqueue_step<double>(c, dt, cap);
}
dh_status dh_finish_steps(dh_ctx* c) { return finish_steps(c, c->host_rec.nstep - c->pending_steps); }

extern "C" dh_status dh_step(dh_ctx* c, double dt, double* dt_used) {
  if (!c) return fail(c, DH_ERR_ARG, "null context");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  const long long before = c->host_rec.nstep - c->pending_steps;
  cudaError_t e = c->prec == DH_F64 ? enqueue_step<double>(c, dt, nullptr) : enqueue_step<float>(c, dt, nullptr);
  if (e != cudaSuccess) return cuda_fail(c, e, "enqueue_step");
  if (dt_used) {
    dh_status s = finish_steps(c, before);
    *dt_used = c->host_rec.dt;
    return s;
  }
  c->host_rec.nstep += 1;  // optimistic host view; corrected by the next finish
  return DH_OK;
}

extern "C" dh_status dh_advance(dh_ctx* c, int n, double* t_out) {
  if (!c) return fail(c, DH_ERR_ARG, "null context");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  if (n < 0) return fail(c, DH_ERR_ARG, "n_steps must be >= 0");
  const long long before = c->host_rec.nstep - c->pending_steps;
  for (int i = 0; i < n; ++i) {
    cudaError_t e = c->prec == DH_F64 ? enqueue_step<double>(c, 0.0, nullptr) : enqueue_step<float>(c, 0.0, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "enqueue_step");
  }
  dh_status s = finish_steps(c, before);
  if (t_out) *t_out = c->host_rec.t;
  return s;
}

extern "C" dh_status dh_get_time(dh_ctx* c, double* t, long long* nstep) {
  if (!c) return fail(c, DH_ERR_ARG, "null context");
  dh_status s = finish_steps(c, c->host_rec.nstep - c->pending_steps);
  if (t) *t = c->host_rec.t;
  if (nstep) *nstep = c->host_rec.nstep;
  return s;
}

extern "C" dh_status dh_compute_dt(dh_ctx* c, double* dt) {
  if (!c || !dt) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  DH_CUDA(c, reset_cfl_bits(c));
  DH_CUDA(c, c->prec == DH_F64 ? cfl_reduce_current<double>(c) : cfl_reduce_current<float>(c));
  unsigned long long bits = 0;
  DH_CUDA(c, cudaMemcpyAsync(&bits, &c->rec->cfl_min_bits, sizeof(bits), cudaMemcpyDeviceToHost,
                             c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  double m;
  if (c->prec == DH_F32) {
    float f;
    unsigned u = (unsigned)bits;
    std::memcpy(&f, &u, 4);
    m = f;
  } else {
    std::memcpy(&m, &bits, 8);
  }
  *dt = std::fmin(c->cfg.cfl * m, c->cfg.dt_max);
  return DH_OK;
}

extern "C" dh_status dh_conserved_totals(dh_ctx* c, double out[5]) {
  if (!c || !out) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  prof_begin(c, DH_KERNEL_REDUCE);
  cudaError_t e = c->prec == DH_F64
      ? launch_totals<double>((const double*)c->U[c->cur], c->n3, c->partials, totals_blocks(), c->totals, c->stream)
      : launch_totals<float>((const float*)c->U[c->cur], c->n3, c->partials, totals_blocks(), c->totals, c->stream);
  prof_end(c, 2);
  if (e != cudaSuccess) return cuda_fail(c, e, "totals");
  DH_CUDA(c, cudaMemcpyAsync(out, c->totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  return DH_OK;
}

static_assert((unsigned)DH_FLAG_NONFINITE == dh::FLAG_NONFINITE &&
                  (unsigned)DH_FLAG_POSITIVITY == dh::FLAG_POSITIVITY &&
                  (unsigned)DH_FLAG_MG_NOCONV == dh::FLAG_MG_NOCONV &&
                  (unsigned)DH_FLAG_COOL_CAP == dh::FLAG_COOL_CAP &&
                  (unsigned)DH_FLAG_TIMEOUT == dh::FLAG_TIMEOUT,
              "public and device status bits");

extern "C" dh_status dh_get_metrics(dh_ctx* c, dh_metrics* out) {
  if (!c || !out) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->initialized) return fail(c, DH_ERR_STATE, "state not initialised");
  // settle enqueued steps (their status is this call's status), then read the record
  dh_status st = finish_steps(c, c->host_rec.nstep - c->pending_steps);
  std::memset(out, 0, sizeof(*out));
  out->t = c->host_rec.t;
  out->dt = c->host_rec.dt;
  out->nstep = c->host_rec.nstep;
  out->flags = c->host_rec.flags;
  out->cool_max_substeps = c->host_rec.cool_nsub_max;
  out->slope_fallbacks = (long long)c->host_rec.slope_fallbacks;
  if (c->cfg.cooling && out->cool_max_substeps < 1 && out->nstep > 0) out->cool_max_substeps = 1;
  dh::mg_last(c, &out->mg_cycles, &out->mg_residual);
  double* mins = c->partials + 2 * totals_blocks();
  cudaError_t e = c->prec == DH_F64
      ? launch_totals<double>((const double*)c->U[c->cur], c->n3, c->partials, totals_blocks(), c->totals, c->stream)
      : launch_totals<float>((const float*)c->U[c->cur], c->n3, c->partials, totals_blocks(), c->totals, c->stream);
  if (e == cudaSuccess)
    e = c->prec == DH_F64
        ? launch_minima<double>((const double*)c->U[c->cur], c->n3, c->cfg.gamma, c->partials, totals_blocks(), mins, c->stream)
        : launch_minima<float>((const float*)c->U[c->cur], c->n3, c->cfg.gamma, c->partials, totals_blocks(), mins, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "metrics");
  double m2[2];
  DH_CUDA(c, cudaMemcpyAsync(out->totals, c->totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  DH_CUDA(c, cudaMemcpyAsync(m2, mins, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  // the substep maximum covers the interval since the previous read
  DH_CUDA(c, cudaMemsetAsync(&c->rec->cool_nsub_max, 0, sizeof(int), c->stream));
  DH_CUDA(c, cudaMemsetAsync(&c->rec->slope_fallbacks, 0, sizeof(unsigned long long), c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  c->host_rec.cool_nsub_max = 0;
  c->host_rec.slope_fallbacks = 0;
  out->rho_min = m2[0];
  out->p_min = m2[1];
  return st;
}

extern "C" dh_status dh_forcing_field(dh_ctx* c, void* a_out, int on_device) {
  if (!c || !a_out) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->cfg.forcing) return fail(c, DH_ERR_STATE, "forcing is off");
  const size_t bytes = (size_t)c->n3 * 3 * esize(c);
  void* dst = a_out;
  if (!on_device) DH_CUDA(c, cudaMalloc(&dst, bytes));
  prof_begin(c, DH_KERNEL_SOURCES);
  cudaError_t e;
  if (c->prec == DH_F64) {
    const double* tw[3] = {(const double*)c->tw[0], (const double*)c->tw[1], (const double*)c->tw[2]};
    e = launch_forcing_field<double>((const double*)c->ahat_norm, tw, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                     (double*)dst, c->stream);
  } else {
    const float* tw[3] = {(const float*)c->tw[0], (const float*)c->tw[1], (const float*)c->tw[2]};
    e = launch_forcing_field<float>((const float*)c->ahat_norm, tw, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                    (float*)dst, c->stream);
  }
  prof_end(c, 1);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(a_out, dst, bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (!on_device) cudaFree(dst);   // on every path: the staging buffer is this call's own
  if (e != cudaSuccess) return cuda_fail(c, e, "forcing_field");
  return DH_OK;
}

extern "C" dh_status dh_forcing_modes(dh_ctx* c, double out[96]) {
  if (!c || !out) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->cfg.forcing) return fail(c, DH_ERR_STATE, "forcing is off");
  DH_CUDA(c, cudaMemcpyAsync(out, c->ahat, 96 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  return DH_OK;
}

extern "C" dh_status dh_set_forcing_modes(dh_ctx* c, const double in[96], int hold) {
  if (!c || !in) return fail(c, DH_ERR_ARG, "null argument");
  if (!c->cfg.forcing) return fail(c, DH_ERR_STATE, "forcing is off");
  DH_CUDA(c, cudaMemcpyAsync(c->ahat, in, 96 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  DH_CUDA(c, cudaStreamSynchronize(c->stream));
  c->ou_hold = hold != 0;
  return DH_OK;
}

extern "C" dh_status dh_profile_enable(dh_ctx* c, int enable) {
  if (!c) return fail(c, DH_ERR_ARG, "null context");
  prof_fold(c);
  for (int k = 0; k < DH_KERNEL_KINDS; ++k) { c->prof_ms[k] = 0.0; c->prof_count[k] = 0; }
  c->prof_on = enable != 0;
  return DH_OK;
}

extern "C" dh_status dh_profile_read(dh_ctx* c, int kind, long long* launches, double* total_ms) {
  if (!c || kind < 0 || kind >= DH_KERNEL_KINDS) return fail(c, DH_ERR_ARG, "bad argument");
  prof_fold(c);
  if (launches) *launches = c->prof_count[kind];
  if (total_ms) *total_ms = c->prof_ms[kind];
  return DH_OK;
}

extern "C" dh_status dh_launch_count(dh_ctx* c, long long* launches) {
  if (!c || !launches) return fail(c, DH_ERR_ARG, "null argument");
  *launches = c->launches;
  return DH_OK;
}

extern "C" const char* dh_last_error(const dh_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

extern "C" const char* dh_status_string(dh_status s) {
  switch (s) {
    case DH_OK: return "DH_OK";
    case DH_ERR_ARG: return "DH_ERR_ARG";
    case DH_ERR_CUDA: return "DH_ERR_CUDA";
    case DH_ERR_NONFINITE: return "DH_ERR_NONFINITE";
    case DH_ERR_POSITIVITY: return "DH_ERR_POSITIVITY";
    case DH_ERR_MG_NOCONV: return "DH_ERR_MG_NOCONV";
    case DH_ERR_STATE: return "DH_ERR_STATE";
  }
  return "unknown";
}
