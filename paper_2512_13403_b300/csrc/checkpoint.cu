// File checkpoints of a context (dh_save / dh_load): everything a continuation depends on, so
// that a loaded context steps bit for bit like the one that was saved.
//
// Layout (native byte order): 8-byte magic "DHCKPT02", a fixed header (geometry, precision,
// physics switches, OU seed and hold flag, gamma and cell widths, t, dt, step count, OU
// normalisation), the OU tables a_hat and its pre-update copy (96 doubles each; forcing only),
// the state (5 planes of the context precision), the potential that warm-starts the next
// Poisson solve as its float-float words (n hi floats, then n lo floats; gravity only), and a
// 64-bit FNV-1a checksum of everything before it.  Version 02 replaced version 01's float64
// potential by the float-float words (same size, other meaning): 01 files are refused.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dh_internal.h"

namespace {

constexpr char kMagic[8] = {'D', 'H', 'C', 'K', 'P', 'T', '0', '2'};

struct CkptHeader {
  int32_t nx, ny, nz, precision;
  int32_t forcing, cooling, gravity, ou_hold;
  uint64_t ou_seed;
  double gamma, dx, dy, dz;
  double t, dt, ou_norm;
  int64_t nstep;
};

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
  h.nx = g.nx; h.ny = g.ny; h.nz = g.nz; h.precision = c->prec;
  h.forcing = g.forcing; h.cooling = g.cooling; h.gravity = g.gravity; h.ou_hold = c->ou_hold;
  h.ou_seed = g.ou_seed;
  h.gamma = g.gamma; h.dx = g.dx; h.dy = g.dy; h.dz = g.dz;
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
  if (h.nx != g.nx || h.ny != g.ny || h.nz != g.nz || h.precision != c->prec ||
      h.forcing != g.forcing || h.cooling != g.cooling || h.gravity != g.gravity ||
      h.ou_seed != g.ou_seed || h.gamma != g.gamma || h.dx != g.dx || h.dy != g.dy || h.dz != g.dz) {
    std::fclose(f);
    return fail(c, DH_ERR_ARG, "dh_load: the checkpoint was written by a different configuration");
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
