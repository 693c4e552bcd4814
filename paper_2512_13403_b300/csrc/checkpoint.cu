// File checkpoints of a context (dh_save / dh_load): everything a continuation depends on, so
// that a loaded context steps bit for bit like the one that was saved.
//
// Layout (native byte order): 8-byte magic "DHCKPT03", a fixed header (every configuration
// field that changes a step: geometry, precision, the scheme, CFL and dt bound, the forcing,
// cooling and multigrid settings; then the OU hold flag, t, dt, step count, OU normalisation),
// the OU tables a_hat and its pre-update copy (96 doubles each; forcing only), the state (5
// planes of the context precision), the potential that warm-starts the next Poisson solve as
// its float-float words (n hi floats, then n lo floats; gravity only), and a 64-bit FNV-1a
// checksum of everything before it.  A file is loaded only into a context whose configuration
// equals the saved one in every field, so that the continuation is the saved run's.  Version
// 03 added the scheme, forcing, cooling and multigrid settings to the header; 01 and 02 files
// are refused.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dh_internal.h"

namespace {

constexpr char kMagic[8] = {'D', 'H', 'C', 'K', 'P', 'T', '0', '3'};

// the configuration fields a step depends on, in a fixed layout
struct CkptConfig {
  int32_t nx, ny, nz, precision;
  int32_t forcing, cooling, gravity, nsub_max;
  int32_t mg_max_cycles, mg_pre, mg_post, mg_smoother;
  int32_t mg_cycle, limiter, integrator, pad;
  uint64_t ou_seed;
  double dx, dy, dz, gamma, cfl, dt_max;
  double ou_tau, ou_arms, t_floor, cool_frac, c_cool;
  double four_pi_G, mg_tol, mg_omega;
};

struct CkptHeader {
  CkptConfig cfg;
  int32_t ou_hold, pad;
  double t, dt, ou_norm;
  int64_t nstep;
};

CkptConfig pack_config(const dh_config& g, int prec) {
  CkptConfig k;
  std::memset(&k, 0, sizeof(k));
  k.nx = g.nx; k.ny = g.ny; k.nz = g.nz; k.precision = prec;
  k.forcing = g.forcing; k.cooling = g.cooling; k.gravity = g.gravity; k.nsub_max = g.nsub_max;
  k.mg_max_cycles = g.mg_max_cycles; k.mg_pre = g.mg_pre; k.mg_post = g.mg_post;
  k.mg_smoother = g.mg_smoother; k.mg_cycle = g.mg_cycle; k.limiter = g.limiter;
  k.integrator = g.integrator;
  k.ou_seed = g.ou_seed;
  k.dx = g.dx; k.dy = g.dy; k.dz = g.dz; k.gamma = g.gamma; k.cfl = g.cfl; k.dt_max = g.dt_max;
  k.ou_tau = g.ou_tau; k.ou_arms = g.ou_arms; k.t_floor = g.t_floor; k.cool_frac = g.cool_frac;
  k.c_cool = g.c_cool; k.four_pi_G = g.four_pi_G; k.mg_tol = g.mg_tol; k.mg_omega = g.mg_omega;
  return k;
}

// The first field in which two configurations differ, or "" (floating-point fields compare
// bit for bit, so that +inf matches +inf).
std::string config_mismatch(const CkptConfig& a, const CkptConfig& b) {
#define DH_CK(f) if (std::memcmp(&a.f, &b.f, sizeof(a.f)) != 0) return #f;
  DH_CK(nx) DH_CK(ny) DH_CK(nz) DH_CK(precision) DH_CK(forcing) DH_CK(cooling) DH_CK(gravity)
  DH_CK(nsub_max) DH_CK(mg_max_cycles) DH_CK(mg_pre) DH_CK(mg_post) DH_CK(mg_smoother)
  DH_CK(mg_cycle) DH_CK(limiter) DH_CK(integrator) DH_CK(ou_seed) DH_CK(dx) DH_CK(dy) DH_CK(dz)
  DH_CK(gamma) DH_CK(cfl) DH_CK(dt_max) DH_CK(ou_tau) DH_CK(ou_arms) DH_CK(t_floor)
  DH_CK(cool_frac) DH_CK(c_cool) DH_CK(four_pi_G) DH_CK(mg_tol) DH_CK(mg_omega)
#undef DH_CK
  return "";
}

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  }
};

dh_status fail(dh_ctx* c, dh_status s, const std::string& m) {
  c->err = m;
  return s;
}

}  // namespace

extern "C" dh_status dh_save(dh_ctx* c, const char* path) {
  if (!c || !path) return DH_ERR_ARG;
  if (!c->initialized) return fail(c, DH_ERR_STATE, "dh_save: state not initialised");
  // settle pending steps so that the host record is the state's
  if (c->pending_steps > 0) {
    dh_status s = dh_finish_steps(c);
    if (s != DH_OK) return s;
  }
  const dh_config& g = c->cfg;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.cfg = pack_config(g, c->prec);
  h.ou_hold = c->ou_hold;
  h.t = c->host_rec.t; h.dt = c->host_rec.dt; h.ou_norm = c->host_rec.ou_norm;
  h.nstep = c->host_rec.nstep;
  std::vector<double> ahat(96, 0.0), ahat_prev(96, 0.0);
  std::vector<unsigned char> state(c->state_bytes);
  std::vector<float> phi;   // float-float words
  cudaError_t e = cudaSuccess;
  if (g.forcing) {
    e = cudaMemcpyAsync(ahat.data(), c->ahat, 96 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ahat_prev.data(), c->ahat_prev, 96 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(state.data(), c->U[c->cur], c->state_bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && g.gravity) {
    phi.resize(2 * (size_t)c->n3);
    e = cudaMemcpyAsync(phi.data(), dh::mg_phi(c), phi.size() * sizeof(float),
                        cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, DH_ERR_CUDA, std::string("dh_save: ") + cudaGetErrorString(e));

  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, DH_ERR_ARG, std::string("dh_save: cannot open ") + path);
  Fnv sum;
  bool ok = true;
  auto put = [&](const void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = std::fwrite(p, 1, n, f) == n;
    sum.add(p, n);
  };
  put(kMagic, sizeof(kMagic));
  put(&h, sizeof(h));
  if (g.forcing) {
    put(ahat.data(), 96 * sizeof(double));
    put(ahat_prev.data(), 96 * sizeof(double));
  }
  put(state.data(), state.size());
  if (g.gravity) put(phi.data(), phi.size() * sizeof(float));
  const uint64_t check = sum.h;
  if (ok) ok = std::fwrite(&check, 1, sizeof(check), f) == sizeof(check);
  if (std::fclose(f) != 0) ok = false;
  if (!ok) return fail(c, DH_ERR_ARG, std::string("dh_save: write failed for ") + path);
  return DH_OK;
}

extern "C" dh_status dh_load(dh_ctx* c, const char* path) {
  if (!c || !path) return DH_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, DH_ERR_ARG, std::string("dh_load: cannot open ") + path);
  Fnv sum;
  bool ok = true;
  auto get = [&](void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) sum.add(p, n);
  };
  char magic[8];
  CkptHeader h;
  get(magic, sizeof(magic));
  get(&h, sizeof(h));
  if (!ok || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) {
    std::fclose(f);
    return fail(c, DH_ERR_ARG, "dh_load: not a checkpoint of this library");
  }
  const dh_config& g = c->cfg;
  const std::string diff = config_mismatch(h.cfg, pack_config(g, c->prec));
  if (!diff.empty()) {
    std::fclose(f);
    return fail(c, DH_ERR_ARG, "dh_load: the checkpoint was written by a different configuration (" +
                                   diff + " differs)");
  }
  std::vector<double> ahat(96), ahat_prev(96);
  std::vector<unsigned char> state(c->state_bytes);
  std::vector<float> phi;   // float-float words
  if (g.forcing) {
    get(ahat.data(), 96 * sizeof(double));
    get(ahat_prev.data(), 96 * sizeof(double));
  }
  get(state.data(), state.size());
  if (g.gravity) {
    phi.resize(2 * (size_t)c->n3);
    get(phi.data(), phi.size() * sizeof(float));
  }
  uint64_t check = 0;
  const uint64_t expect = sum.h;
  if (ok) ok = std::fread(&check, 1, sizeof(check), f) == sizeof(check);
  std::fclose(f);
  if (!ok) return fail(c, DH_ERR_ARG, "dh_load: the file is truncated");
  if (check != expect) return fail(c, DH_ERR_ARG, "dh_load: checksum mismatch");

  dh::StepRecord r;
  std::memset(&r, 0, sizeof(r));
  r.t = h.t;
  r.dt = h.dt;
  r.nstep = h.nstep;
  r.ou_norm = h.ou_norm;
  r.fail_step = -1;
  r.cfl_min_bits = c->prec == DH_F32 ? (unsigned long long)0x7f800000u : 0x7ff0000000000000ull;
  cudaError_t e = cudaMemcpyAsync(c->U[0], state.data(), c->state_bytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && g.forcing) {
    e = cudaMemcpyAsync(c->ahat, ahat.data(), 96 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->ahat_prev, ahat_prev.data(), 96 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess && g.gravity)
    e = cudaMemcpyAsync(dh::mg_phi(c), phi.data(), phi.size() * sizeof(float),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // host vectors go out of scope
  if (e != cudaSuccess) return fail(c, DH_ERR_CUDA, std::string("dh_load: ") + cudaGetErrorString(e));
  c->cur = 0;
  c->pending_steps = 0;
  c->host_rec = r;
  c->ou_hold = h.ou_hold;
  c->initialized = true;
  dh_status s = dh_refresh_cfl(c);
  if (s != DH_OK) return s;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, DH_ERR_CUDA, std::string("dh_load: ") + cudaGetErrorString(e));
  return DH_OK;
}
