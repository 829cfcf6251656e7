// C ABI of the library (declared in include/mqs.h): context and handle
// management, the mesh pattern build, batch set-up, the propagate driver for
// sequential and Parareal time stepping, readouts and the MLMC estimator.
#include "mqs_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>

namespace mqs {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches += n; }

namespace {

constexpr double kTwoPi = 6.28318530717958647692;
constexpr int kReplaceEvery = 50;

enum { V_A0, V_A1, V_Y, V_R, V_P, V_Q, V_Z, V_B, kNV64 };
enum { W_P32, W_Q32, kNV32 };

struct ValueSet {
  double dt = 0.0;
  DevBuf A, A32, Dinv;
};

struct FactorSet {
  double dt = 0.0;
  bool have64 = false, have32 = false, have_cpl = false;
  DevBuf LB, invd, Binv, bad;   // [samples][n][bw+1], [samples][n], [samples][n/32][32][32], [samples]
  DevBuf B64, B64T, C1, C2, D1, D2;   // [samples][n/64][64][64] block inverses and couplings (cluster kernels)
  DevBuf LBf, invdf, Binvf;     // FP32 factor (mixed precision)
};

// Lanes of the banded direct solver: one CTA per lane, vectors lane-major.
struct DirectSet {
  int lanes = 0, n = 0;
  DevBuf vec, qraw, status, desc;
  std::vector<DirectLane> host;
  int ensure(int lanes_, int n_) {
    lanes = lanes_;
    n = n_;
    MQS_TRY(vec.ensure((size_t)lanes * 5 * n * sizeof(double)));
    MQS_TRY(qraw.ensure((size_t)lanes * sizeof(double)));
    MQS_TRY(status.ensure((size_t)lanes * sizeof(int32_t)));
    return MQS_OK;
  }
  // vectors of a lane: 0 a0, 1 a1, 2 y, 3 work (permuted), 4 b (mixed)
  double* v(int lane, int j) const { return vec.as<double>() + ((size_t)lane * 5 + j) * n; }
};

struct LaneSet {
  int lanes = 0;
  int64_t xs = 0;
  int n = 0;
  DevBuf v64, v32, amp, phi, k0, qraw, status, iters, tiles;
  std::vector<TileDesc> host_tiles;
  int ensure(int lanes_, int64_t xs_, int n_, bool mixed) {
    lanes = lanes_;
    xs = xs_;
    n = n_;
    const size_t per = (size_t)n * (size_t)xs;
    MQS_TRY(v64.ensure(per * kNV64 * sizeof(double)));
    if (mixed) MQS_TRY(v32.ensure(per * kNV32 * sizeof(float)));
    MQS_TRY(amp.ensure((size_t)xs * kMaxPhases * sizeof(double)));
    MQS_TRY(phi.ensure((size_t)xs * kMaxPhases * sizeof(double)));
    MQS_TRY(k0.ensure((size_t)xs * sizeof(int32_t)));
    MQS_TRY(qraw.ensure((size_t)xs * sizeof(double)));
    MQS_TRY(status.ensure((size_t)xs * sizeof(int32_t)));
    MQS_TRY(iters.ensure((size_t)xs * sizeof(double)));
    return MQS_OK;
  }
  double* vec(int j) const { return v64.as<double>() + (size_t)j * n * xs; }
  float* vec32(int j) const { return v32.p ? v32.as<float>() + (size_t)j * n * xs : nullptr; }
  LaneArrays arrays() const {
    return LaneArrays{amp.as<double>(), phi.as<double>(), k0.as<int32_t>(), qraw.as<double>(),
                      status.as<int32_t>(), iters.as<double>()};
  }
};

// Pinned host memory mapped into the device address space (written by
// kernels, read by the host without a copy, and the reverse).
struct MappedBuf {
  void* h = nullptr;
  void* d = nullptr;
  size_t bytes = 0;
  MappedBuf() = default;
  MappedBuf(const MappedBuf&) = delete;
  MappedBuf& operator=(const MappedBuf&) = delete;
  ~MappedBuf() {
    if (h) cudaFreeHost(h);
  }
  int ensure(size_t n) {
    if (n <= bytes && h) return MQS_OK;
    if (h) cudaFreeHost(h);
    h = d = nullptr;
    bytes = 0;
    MQS_CUDA_TRY(cudaHostAlloc(&h, n, cudaHostAllocMapped));
    MQS_CUDA_TRY(cudaHostGetDevicePointer(&d, h, 0));
    bytes = n;
    return MQS_OK;
  }
};

struct Batch {
  int mesh_id = -1;
  int n = 0, n_params = 0;
  DevBuf params;
  bool time_set = false;
  double t0 = 0.0, t_end = 0.0, freq = 50.0;
  int qoi_kind = MQS_QOI_JOULE;
  DevBuf Mv, Kv;
  bool have_M = false, have_K = false;
  std::vector<std::unique_ptr<ValueSet>> vsets;
  LaneSet plain, par, chain;
  int nf_pad = 0, nc_pad = 0;
  bool has_coarse = false;
  DevBuf U, G, jump2, norm2;
  int mode = 0;      // 0 nothing run, 1 sequential, 2 Parareal
  int M = 0;
  DevBuf qoi, status;
  int level = 0;
  double stats[MQS_N_STATS] = {};
  // banded direct solver
  int solver = MQS_SOLVER_PCG;
  std::vector<double> hparams;                 // host copy of the parameters
  std::vector<std::unique_ptr<FactorSet>> fsets;
  DirectSet dplain, dpar, dchain;
  DevBuf E;                                    // Parareal fine ends, lane-major
  double* E_final = nullptr;                   // fine ends of the last Parareal iteration
  DevBuf qraw2, pdesc;                         // pipelined Parareal: [2][lanes] QoI partials,
                                               // [2][lanes] fine-lane descriptors
  MappedBuf jhist, nhist, stop;                // per-iteration jump / norm squares, cancel word
  int nf_direct = 0;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // side stream for work that overlaps the main stream (Parareal: the fine
  // factorisation runs beside the coarse one and the first coarse sweep)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_comp0 = nullptr, ev_comp1 = nullptr;   // companion solve beside Parareal
  int n_sm = 1;
  int test_hook = 0;   // MQS_TEST_HOOK_* of mqs_set_test_hook
  std::vector<std::unique_ptr<MeshDev>> meshes;
  std::vector<std::unique_ptr<Batch>> batches;
  DevBuf mlmc;
  int n_levels = 0;
  // pipelined Parareal: streams of the fine chunks and the events that order
  // them against the sweep chunks ([iteration parity][chunk])
  std::vector<cudaStream_t> fine_st;
  std::vector<cudaEvent_t> ev_sweep[2], ev_fine[2], ev_fjoin;
  // instrumentation: event pairs around the stepping (0) and coarse-sweep (1)
  // launches, on the stream of each launch; t0 on the main stream when enabled
  bool prof = false;
  cudaEvent_t prof_t0 = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[2];
  size_t ev_used[2] = {0, 0};
  ~Ctx() {
    for (auto& v : ev)
      for (auto& e : v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
    if (prof_t0) cudaEventDestroy(prof_t0);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    for (cudaStream_t f : fine_st) {
      cudaStreamSynchronize(f);
      cudaStreamDestroy(f);
    }
    for (int p = 0; p < 2; ++p) {
      for (cudaEvent_t e : ev_sweep[p]) cudaEventDestroy(e);
      for (cudaEvent_t e : ev_fine[p]) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : ev_fjoin) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_comp0) cudaEventDestroy(ev_comp0);
    if (ev_comp1) cudaEventDestroy(ev_comp1);
  }
};

// `chunks` streams for the fine chunks and the ordering events.
int ensure_pipeline(Ctx& c, int chunks) {
  while ((int)c.fine_st.size() < chunks) {
    cudaStream_t f;
    MQS_CUDA_TRY(cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking));
    c.fine_st.push_back(f);
    cudaEvent_t e;
    MQS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c.ev_fjoin.push_back(e);
    for (int p = 0; p < 2; ++p) {
      MQS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c.ev_sweep[p].push_back(e);
      MQS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c.ev_fine[p].push_back(e);
    }
  }
  return MQS_OK;
}



int ensure_side(Ctx& c) {
  if (!c.side) MQS_CUDA_TRY(cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking));
  if (!c.ev_fork) MQS_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
  if (!c.ev_join) MQS_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
  if (!c.ev_comp0) MQS_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_comp0, cudaEventDisableTiming));
  if (!c.ev_comp1) MQS_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_comp1, cudaEventDisableTiming));
  return MQS_OK;
}

// Work issued while one of these is alive goes to the context's side stream.
struct OnSide {
  Ctx& c;
  cudaStream_t saved;
  explicit OnSide(Ctx& c_) : c(c_), saved(c_.stream) { c.stream = c.side; }
  ~OnSide() { c.stream = saved; }
};

// Record the start (begin = true) or end event of a launch of kind k on
// stream st (default: the context's stream).
int prof_mark(Ctx& c, int k, bool begin, cudaStream_t st = nullptr) {
  if (!c.prof) return MQS_OK;
  if (!st) st = c.stream;
  if (begin) {
    if (c.ev_used[k] == c.ev[k].size()) {
      cudaEvent_t a, b;
      MQS_CUDA_TRY(cudaEventCreate(&a));
      MQS_CUDA_TRY(cudaEventCreate(&b));
      c.ev[k].emplace_back(a, b);
    }
    MQS_CUDA_TRY(cudaEventRecord(c.ev[k][c.ev_used[k]].first, st));
  } else {
    MQS_CUDA_TRY(cudaEventRecord(c.ev[k][c.ev_used[k]].second, st));
    c.ev_used[k]++;
  }
  return MQS_OK;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace mqs

struct mqs_ctx {
  mqs::Ctx c;
};

using namespace mqs;

namespace mqs {
// Accessors for other translation units of the library (the request server).
const MeshDev* ctx_mesh(mqs_ctx* ctx, int id) {
  if (!ctx || id < 0 || id >= (int)ctx->c.meshes.size() || !ctx->c.meshes[id]) return nullptr;
  return ctx->c.meshes[id].get();
}
int ctx_device(mqs_ctx* ctx) { return ctx->c.device; }
}  // namespace mqs

namespace {

int enter(mqs_ctx* ctx) {
  clear_error();
  if (!ctx) {
    set_error("null context");
    return MQS_EINVAL;
  }
  MQS_CUDA_TRY(cudaSetDevice(ctx->c.device));
  return MQS_OK;
}

MeshDev* get_mesh(mqs_ctx* ctx, int id) {
  if (id < 0 || id >= (int)ctx->c.meshes.size() || !ctx->c.meshes[id]) {
    set_error("invalid mesh id %d", id);
    return nullptr;
  }
  return ctx->c.meshes[id].get();
}

Batch* get_batch(mqs_ctx* ctx, int id) {
  if (id < 0 || id >= (int)ctx->c.batches.size() || !ctx->c.batches[id]) {
    set_error("invalid batch id %d", id);
    return nullptr;
  }
  return ctx->c.batches[id].get();
}

// Lane-tile width L and cluster size C for `lanes` lanes over n rows.  A team
// lives for the whole run, so all teams should be resident at once: among the
// tile widths whose tiles fit the resident cluster count for some C, take the
// shape that keeps the most CTAs busy (ties: wider tiles), with at least one
// full pass of row slots per CTA.  When the tiles outnumber the resident
// clusters even at C = 1, the widest tile and C = 1 are used (several waves).
void choose_shape(const Ctx& c, int lanes, int n, int precision, int max_L, int& L, int& C) {
  const int forced_L = env_int("MQS_TILE_L", 0);
  const int forced_C = env_int("MQS_CLUSTER", 0);
  int best_L = 0, best_C = 0;
  int64_t best_busy = -1;
  int lanes_p2 = 1;
  while (lanes_p2 < lanes && lanes_p2 < 32) lanes_p2 <<= 1;
  for (int cand = 32; cand >= 1; cand >>= 1) {
    if (cand > max_L) continue;
    if (forced_L > 0 ? cand != forced_L : cand > lanes_p2) continue;
    const int tiles = (lanes + cand - 1) / cand;
    const int rows_pass = team_threads() / cand;
    const int c_rows = std::max(1, n / rows_pass);
    const int cmax = std::min(max_cluster(cand, precision, c.n_sm), c_rows);
    for (int cc = cmax; cc >= 1; --cc) {
      if (forced_C > 0 && cc != std::min(forced_C, cmax)) continue;
      const int active = max_active_clusters(cand, precision, cc);
      if (active < tiles && !(forced_C > 0)) continue;
      const int64_t busy = (int64_t)std::min(tiles, std::max(active, 1)) * cc;
      if (busy > best_busy) {
        best_busy = busy;
        best_L = cand;
        best_C = cc;
      }
      break;   // the largest C that fits is the best for this width
    }
  }
  if (best_L == 0) {
    // more tiles than resident clusters: widest tile, single-CTA teams
    best_L = std::min(max_L, forced_L > 0 ? forced_L : lanes_p2);
    best_C = forced_C > 0 ? std::min(forced_C, max_cluster(best_L, precision, c.n_sm)) : 1;
  }
  L = best_L;
  C = std::max(1, best_C);
}

ValueSet* value_set(mqs_ctx* ctx, Batch& b, const MeshDev& m, double dt, bool mixed, int& rc) {
  rc = MQS_OK;
  ValueSet* vs = nullptr;
  for (auto& v : b.vsets)
    if (v->dt == dt) vs = v.get();
  const int64_t nnz = m.nnz;
  const cudaStream_t st = ctx->c.stream;
  if (!vs) {
    b.vsets.emplace_back(new ValueSet());
    vs = b.vsets.back().get();
    vs->dt = dt;
    if ((rc = vs->A.ensure((size_t)nnz * b.n * sizeof(double))) != MQS_OK) return nullptr;
    if ((rc = vs->Dinv.ensure((size_t)m.n_free * b.n * sizeof(double))) != MQS_OK) return nullptr;
    rc = expand_values(m, b.params.as<double>(), b.n, b.n_params, dt, b.n, vs->A.as<double>(),
                       nullptr, nullptr, nullptr, vs->Dinv.as<double>(), nullptr, b.n, st);
    if (rc != MQS_OK) return nullptr;
  }
  if (mixed && !vs->A32.p) {
    if ((rc = vs->A32.ensure((size_t)nnz * b.n * sizeof(float))) != MQS_OK) return nullptr;
    rc = expand_values(m, b.params.as<double>(), b.n, b.n_params, dt, b.n, nullptr, nullptr,
                       nullptr, vs->A32.as<float>(), nullptr, nullptr, b.n, st);
    if (rc != MQS_OK) return nullptr;
  }
  return vs;
}

int ensure_mk(mqs_ctx* ctx, Batch& b, const MeshDev& m) {
  const cudaStream_t st = ctx->c.stream;
  if (!b.have_M) {
    MQS_TRY(b.Mv.ensure((size_t)m.nnz * b.n * sizeof(double)));
    MQS_TRY(expand_values(m, b.params.as<double>(), b.n, b.n_params, 1.0, b.n, nullptr,
                          b.Mv.as<double>(), nullptr, nullptr, nullptr, nullptr, b.n, st));
    b.have_M = true;
  }
  if (b.qoi_kind == MQS_QOI_ENERGY && !b.have_K) {
    MQS_TRY(b.Kv.ensure((size_t)m.nnz * b.n * sizeof(double)));
    MQS_TRY(expand_values(m, b.params.as<double>(), b.n, b.n_params, 1.0, b.n, nullptr, nullptr,
                          b.Kv.as<double>(), nullptr, nullptr, nullptr, b.n, st));
    b.have_K = true;
  }
  return MQS_OK;
}

TileDesc make_tile(const LaneSet& ls, int lane0, int n_active, const ValueSet& v, const Batch& b,
                   int value_col, int per_lane_values, double dt, int n_steps, int init_from_a0,
                   bool mixed) {
  TileDesc t;
  memset(&t, 0, sizeof(t));
  t.A = v.A.as<double>() + value_col;
  t.M = b.Mv.as<double>() + value_col;
  t.K = b.have_K && b.qoi_kind == MQS_QOI_ENERGY ? b.Kv.as<double>() + value_col : nullptr;
  t.A32 = mixed ? v.A32.as<float>() + value_col : nullptr;
  t.Dinv = v.Dinv.as<double>() + value_col;
  t.vs = b.n;
  t.ds = b.n;
  t.ls = per_lane_values;
  t.lane0 = lane0;
  t.a0 = ls.vec(V_A0) + lane0;
  t.a1 = ls.vec(V_A1) + lane0;
  t.y = ls.vec(V_Y) + lane0;
  t.r = ls.vec(V_R) + lane0;
  t.p = ls.vec(V_P) + lane0;
  t.q = ls.vec(V_Q) + lane0;
  t.z = ls.vec(V_Z) + lane0;
  t.b = mixed ? ls.vec(V_B) + lane0 : nullptr;
  t.p32 = mixed ? ls.vec32(W_P32) + lane0 : nullptr;
  t.q32 = mixed ? ls.vec32(W_Q32) + lane0 : nullptr;
  t.xs = ls.xs;
  t.dt = dt;
  t.t0 = b.t0;
  t.n_steps = n_steps;
  t.n_active = n_active;
  t.init_from_a0 = init_from_a0;
  return t;
}

int upload_tiles(mqs_ctx* ctx, LaneSet& ls) {
  MQS_TRY(ls.tiles.ensure(std::max<size_t>(1, ls.host_tiles.size()) * sizeof(TileDesc)));
  if (!ls.host_tiles.empty())
    MQS_CUDA_TRY(cudaMemcpyAsync(ls.tiles.p, ls.host_tiles.data(),
                                 ls.host_tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice,
                                 ctx->c.stream));
  return MQS_OK;
}

TeamConst team_const(const MeshDev& m, const Batch& b, const LaneSet& ls, double cg_tol,
                     int cg_max) {
  TeamConst kc;
  memset(&kc, 0, sizeof(kc));
  kc.rowptr = m.rowptr.as<int32_t>();
  kc.colidx = m.colidx.as<int32_t>();
  kc.F = m.F.as<double>();
  kc.n = m.n_free;
  kc.n_phases = m.n_phases;
  kc.qoi_kind = b.qoi_kind;
  kc.max_it = cg_max;
  kc.replace_every = kReplaceEvery;
  kc.tol2 = cg_tol * cg_tol;
  kc.omega = kTwoPi * b.freq;
  kc.lanes = ls.arrays();
  return kc;
}

int steps_of(double T, double dt, int& n_steps) {
  if (!(dt > 0.0) || !std::isfinite(dt)) {
    set_error("step size must be positive and finite (got %g)", dt);
    return MQS_EINVAL;
  }
  const double q = T / dt;
  const double r = std::nearbyint(q);
  if (r < 1.0 || std::fabs(q - r) > 1e-9 * std::max(1.0, r) || r > 2e9) {
    set_error("(t_end - t0) / dt = %.12g is not a positive integer", q);
    return MQS_EINVAL;
  }
  n_steps = (int)r;
  return MQS_OK;
}

double qoi_scale(int kind, int n_steps, double dt) {
  return kind == MQS_QOI_JOULE ? 1.0 / ((double)n_steps * dt) : 1.0 / (double)n_steps;
}

// Sequential solves: `segments` sets of n lanes each (fine, and coarse if vc).
int run_plain(mqs_ctx* ctx, Batch& b, const MeshDev& m, const ValueSet* vf, int nsf,
              const ValueSet* vc, int nsc, int precision, double cg_tol, int cg_max) {
  const bool mixed = precision == MQS_MIXED;
  const int nf = vf ? b.n : 0, nc = vc ? b.n : 0;
  int L, C;
  choose_shape(ctx->c, nf + nc, m.n_free, precision, 32, L, C);
  b.nf_pad = (int)round_up(nf, L);
  b.nc_pad = (int)round_up(nc, L);
  const int64_t xs = b.nf_pad + b.nc_pad;
  LaneSet& ls = b.plain;
  MQS_TRY(ls.ensure((int)xs, xs, m.n_free, mixed));
  const cudaStream_t st = ctx->c.stream;
  MQS_CUDA_TRY(cudaMemsetAsync(ls.k0.p, 0, xs * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(ls.qraw.p, 0, xs * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(ls.status.p, 0, xs * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(ls.iters.p, 0, xs * sizeof(double), st));
  ls.host_tiles.clear();
  if (nf) {
    MQS_TRY(lane_sources(b.params.as<double>(), b.n, b.n_params, m.n_regions, m.n_phases, 1,
                         ls.amp.as<double>(), ls.phi.as<double>(), st));
    for (int l0 = 0; l0 < nf; l0 += L)
      ls.host_tiles.push_back(make_tile(ls, l0, std::min(L, nf - l0), *vf, b, l0, 1, vf->dt, nsf,
                                        0, mixed));
  }
  if (nc) {
    MQS_TRY(lane_sources(b.params.as<double>(), b.n, b.n_params, m.n_regions, m.n_phases, 1,
                         ls.amp.as<double>() + (size_t)b.nf_pad * kMaxPhases,
                         ls.phi.as<double>() + (size_t)b.nf_pad * kMaxPhases, st));
    for (int l0 = 0; l0 < nc; l0 += L)
      ls.host_tiles.push_back(make_tile(ls, b.nf_pad + l0, std::min(L, nc - l0), *vc, b, l0, 1,
                                        vc->dt, nsc, 0, mixed));
  }
  MQS_TRY(upload_tiles(ctx, ls));
  const TeamConst kc = team_const(m, b, ls, cg_tol, cg_max);
  MQS_TRY(prof_mark(ctx->c, 0, true));
  MQS_TRY(launch_propagate(ls.tiles.as<TileDesc>(), (int)ls.host_tiles.size(), L, C, precision,
                           kc, st));
  MQS_TRY(prof_mark(ctx->c, 0, false));
  b.stats[6] += (double)nf * nsf + (double)nc * nsc;
  b.stats[1] += (double)nf * nsf + (double)nc * nsc;
  b.stats[2] += (double)nf * nsf + (double)nc * nsc;
  return MQS_OK;
}

int sum_host(mqs_ctx* ctx, const DevBuf& buf, int64_t count, double& out) {
  std::vector<double> h((size_t)count);
  if (count)
    MQS_CUDA_TRY(cudaMemcpyAsync(h.data(), buf.p, count * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->c.stream));
  MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  out = 0.0;
  for (double v : h) out += v;
  return MQS_OK;
}

int run_parareal(mqs_ctx* ctx, Batch& b, const MeshDev& m, const ValueSet& vf,
                 const ValueSet& vcoarse, int n_steps, int M, int cf, int max_iters, double tol,
                 int precision, double cg_tol, int cg_max, int& iters_out) {
  const bool mixed = precision == MQS_MIXED;
  const cudaStream_t st = ctx->c.stream;
  const int S = n_steps / M, Sc = S / cf;
  const int ns = b.n;
  const int lanes = ns * M;
  int maxL = 1;
  while (maxL * 2 <= 32 && M % (maxL * 2) == 0) maxL *= 2;
  int Lf, Cf;
  choose_shape(ctx->c, lanes, m.n_free, precision, maxL, Lf, Cf);
  LaneSet& pf = b.par;
  MQS_TRY(pf.ensure(lanes, lanes, m.n_free, mixed));
  int Lc, Cc;
  choose_shape(ctx->c, ns, m.n_free, precision, 32, Lc, Cc);
  const int64_t xs_c = round_up(ns, Lc);
  LaneSet& pc = b.chain;
  MQS_TRY(pc.ensure((int)xs_c, xs_c, m.n_free, mixed));
  const size_t field = (size_t)m.n_free * lanes * sizeof(double);
  MQS_TRY(b.U.ensure(field));
  MQS_TRY(b.G.ensure(field));
  MQS_TRY(b.jump2.ensure((size_t)ns * M * sizeof(double)));
  MQS_TRY(b.norm2.ensure((size_t)ns * M * sizeof(double)));
  MQS_CUDA_TRY(cudaMemsetAsync(b.U.p, 0, field, st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.G.p, 0, field, st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.norm2.p, 0, (size_t)ns * M * sizeof(double), st));
  // fine lanes: lane = sample * M + slice, k0 = slice * S
  MQS_TRY(lane_sources(b.params.as<double>(), ns, b.n_params, m.n_regions, m.n_phases, M,
                       pf.amp.as<double>(), pf.phi.as<double>(), st));
  MQS_TRY(fill_k0(pf.k0.as<int32_t>(), lanes, M, S, st));
  MQS_CUDA_TRY(cudaMemsetAsync(pf.qraw.p, 0, lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(pf.status.p, 0, lanes * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(pf.iters.p, 0, lanes * sizeof(double), st));
  // chain lanes: one per sample
  MQS_TRY(lane_sources(b.params.as<double>(), ns, b.n_params, m.n_regions, m.n_phases, 1,
                       pc.amp.as<double>(), pc.phi.as<double>(), st));
  MQS_CUDA_TRY(cudaMemsetAsync(pc.k0.p, 0, xs_c * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(pc.status.p, 0, xs_c * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(pc.iters.p, 0, xs_c * sizeof(double), st));
  pc.host_tiles.clear();
  for (int l0 = 0; l0 < ns; l0 += Lc)
    pc.host_tiles.push_back(make_tile(pc, l0, std::min(Lc, ns - l0), vcoarse, b, l0, 1,
                                      vcoarse.dt, Sc, 1, mixed));
  MQS_TRY(upload_tiles(ctx, pc));
  const TeamConst kcc = team_const(m, b, pc, cg_tol, cg_max);
  ChainDesc ch;
  ch.U = b.U.as<double>();
  ch.E = pf.vec(V_A0);
  ch.G = b.G.as<double>();
  ch.xs_par = lanes;
  ch.M = M;
  ch.steps_per_slice = Sc;
  ch.jump2 = b.jump2.as<double>();
  ch.norm2 = b.norm2.as<double>();
  // k = 0: coarse sweep
  ch.s_begin = 0;
  ch.first_sweep = 1;
  MQS_CUDA_TRY(cudaMemsetAsync(b.jump2.p, 0, (size_t)ns * M * sizeof(double), st));
  MQS_TRY(prof_mark(ctx->c, 1, true));
  MQS_TRY(launch_chain(pc.tiles.as<TileDesc>(), (int)pc.host_tiles.size(), Lc, Cc, precision,
                       kcc, ch, st));
  MQS_TRY(prof_mark(ctx->c, 1, false));
  double exec_steps = (double)ns * (M - 1) * Sc;
  double chain_steps = (double)ns * (M - 1) * Sc, fine_steps = 0.0;
  std::vector<double> hj((size_t)ns * M), hn((size_t)ns * M);
  int k = 0;
  for (k = 1; k <= max_iters; ++k) {
    // fine propagation of slices k-1 .. M-1 (pruned at tile granularity)
    MQS_TRY(copy_lanes(b.U.as<double>(), pf.vec(V_A0), m.n_free, lanes, 0, lanes, 0, 0, st));
    pf.host_tiles.clear();
    for (int s = 0; s < ns; ++s)
      for (int j0 = 0; j0 < M; j0 += Lf) {
        if (j0 + Lf <= k - 1) continue;
        pf.host_tiles.push_back(make_tile(pf, s * M + j0, Lf, vf, b, s, 0, vf.dt, S, 1, mixed));
        exec_steps += (double)Lf * S;
        fine_steps += (double)Lf * S;
      }
    MQS_TRY(upload_tiles(ctx, pf));
    const TeamConst kcf = team_const(m, b, pf, cg_tol, cg_max);
    MQS_TRY(prof_mark(ctx->c, 0, true));
    MQS_TRY(launch_propagate(pf.tiles.as<TileDesc>(), (int)pf.host_tiles.size(), Lf, Cf,
                             precision, kcf, st));
    MQS_TRY(prof_mark(ctx->c, 0, false));
    // coarse sweep with the Eq. 12 correction on slices k-1 .. M-2
    MQS_CUDA_TRY(cudaMemsetAsync(b.jump2.p, 0, (size_t)ns * M * sizeof(double), st));
    if (k - 1 <= M - 2) {
      ch.s_begin = k - 1;
      ch.first_sweep = 0;
      MQS_TRY(prof_mark(ctx->c, 1, true));
      MQS_TRY(launch_chain(pc.tiles.as<TileDesc>(), (int)pc.host_tiles.size(), Lc, Cc, precision,
                           kcc, ch, st));
      MQS_TRY(prof_mark(ctx->c, 1, false));
      exec_steps += (double)ns * (M - 1 - (k - 1)) * Sc;
      chain_steps += (double)ns * (M - 1 - (k - 1)) * Sc;
    }
    MQS_CUDA_TRY(cudaMemcpyAsync(hj.data(), b.jump2.p, hj.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    MQS_CUDA_TRY(cudaMemcpyAsync(hn.data(), b.norm2.p, hn.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    MQS_CUDA_TRY(cudaStreamSynchronize(st));
    bool all = true;
    for (int s = 0; s < ns; ++s) {
      double num = 0.0, den = 0.0;
      for (int j = 0; j < M; ++j) {
        num = std::max(num, std::sqrt(hj[(size_t)s * M + j]));
        den = std::max(den, std::sqrt(hn[(size_t)s * M + j]));
      }
      const double jump = den > 0.0 ? num / den : num;
      if (!(jump <= tol)) all = false;
    }
    if (all || k >= M) break;
  }
  iters_out = std::min(k, max_iters);
  b.stats[1] += exec_steps;
  b.stats[6] += fine_steps;
  b.stats[7] += chain_steps;
  b.stats[2] += (double)ns * n_steps;
  return MQS_OK;
}


FactorSet* factor_set(mqs_ctx* ctx, Batch& b, const MeshDev& m, double dt, bool mixed, int& rc) {
  rc = MQS_OK;
  FactorSet* f = nullptr;
  for (auto& x : b.fsets)
    if (x->dt == dt) f = x.get();
  if (f && (mixed ? f->have32 : f->have64)) return f;
  ValueSet* v = value_set(ctx, b, m, dt, false, rc);
  if (!v) return nullptr;
  if (!f) {
    b.fsets.emplace_back(new FactorSet());
    f = b.fsets.back().get();
    f->dt = dt;
  }
  const size_t fstride = (size_t)m.n_free * (m.bw + 1);
  const size_t bstride = (size_t)block_count(m.n_free) * 32 * 32;
  if ((rc = f->bad.ensure((size_t)b.n * sizeof(int32_t))) != MQS_OK) return nullptr;
  if (mixed) {
    if ((rc = f->LBf.ensure(fstride * b.n * sizeof(float))) != MQS_OK) return nullptr;
    if ((rc = f->invdf.ensure((size_t)m.n_free * b.n * sizeof(float))) != MQS_OK) return nullptr;
    if ((rc = f->Binvf.ensure(bstride * b.n * sizeof(float))) != MQS_OK) return nullptr;
    rc = band_factor<float>(m, v->A.as<double>(), b.n, b.n, f->LBf.as<float>(),
                            f->invdf.as<float>(), f->Binvf.as<float>(), f->bad.as<int32_t>(),
                            ctx->c.stream);
    f->have32 = rc == MQS_OK;
  } else {
    if ((rc = f->LB.ensure(fstride * b.n * sizeof(double))) != MQS_OK) return nullptr;
    if ((rc = f->invd.ensure((size_t)m.n_free * b.n * sizeof(double))) != MQS_OK) return nullptr;
    if ((rc = f->Binv.ensure(bstride * b.n * sizeof(double))) != MQS_OK) return nullptr;
    rc = band_factor<double>(m, v->A.as<double>(), b.n, b.n, f->LB.as<double>(),
                             f->invd.as<double>(), f->Binv.as<double>(), f->bad.as<int32_t>(),
                             ctx->c.stream);
    f->have64 = rc == MQS_OK;
  }
  if (rc == MQS_OK && !mixed) f->have_cpl = false;   // new factor: couplings are stale
  return rc == MQS_OK ? f : nullptr;
}

// Elements per factor of each block array of the cluster kernels.
size_t cluster_bstride(const MeshDev& m) {
  const size_t kb = (size_t)cluster_block_rows();
  return ((size_t)m.n_free + kb - 1) / kb * kb * kb;
}

// Block inverses and couplings of an FP64 factor set, for the cluster stepping kernels.
int ensure_couplings(mqs_ctx* ctx, Batch& b, const MeshDev& m, FactorSet& f) {
  if (f.have_cpl) return MQS_OK;
  const size_t bstride = cluster_bstride(m);
  for (DevBuf* x : {&f.B64, &f.B64T, &f.C1, &f.C2, &f.D1, &f.D2})
    MQS_TRY(x->ensure(bstride * b.n * sizeof(double)));
  MQS_TRY(block_prep(m, b.n, f.LB.as<double>(), f.B64.as<double>(), f.B64T.as<double>(),
                     f.C1.as<double>(), f.C2.as<double>(), f.D1.as<double>(), f.D2.as<double>(),
                     ctx->c.stream));
  f.have_cpl = true;
  return MQS_OK;
}

// Cluster size of the FP64 stepping kernels (each CTA keeps its own rows of
// the work vector and a ring of recently solved rows in shared memory); 0
// selects the one-CTA kernels of mqs_direct.cu (mixed precision, and batches
// of at least two lanes per SM whose work vectors live in L2).  The widest
// split (8, 4, 2 CTAs per lane) whose clusters all fit the SMs in one wave;
// with more lanes, the narrowest split that fits shared memory (2 on the 20k
// annulus, 4 on the 80k annulus) in several waves.  Meshes too large for a
// one-CTA work vector in shared memory always take the cluster kernels.
// Measured on the 20k-node annulus: one lane (the coarse sweep) steps fastest
// on 8 CTAs; 64 lanes on 2 CTAs each (2.55 ms per step); the one-CTA form of
// these kernels (8 ms per step) and the one-CTA kernel of mqs_direct.cu (7 ms)
// lose to 2 CTAs per lane even at two waves.
// env MQS_DIRECT_CLUSTER=0/1/2/4/8 forces a choice.
int direct_cluster(const MeshDev& m, int lanes, int n_sm, bool mixed, bool wide) {
  if (mixed) return 0;
  const int n = m.n_free, bw = m.bw;
  const int forced = env_int("MQS_DIRECT_CLUSTER", -1);
  if (forced == 0) return 0;
  if ((forced == 1 || forced == 2 || forced == 4 || forced == 8) && cluster_fits(n, bw, forced))
    return forced;
  const bool big = n > direct_smem_max_n(0);
  if (!wide && !big) return 0;
  for (int cl : {8, 4, 2})
    if (lanes * cl <= n_sm && lanes <= cluster_max_active(cl, n, bw)) return cl;
  for (int cl : {2, 4, 8})
    if (cluster_max_active(cl, n, bw) > 0) return cl;
  return 0;
}

// lanes: CTAs of the launch; big batches run 256-thread CTAs with the work
// vector in L2, several per SM (env MQS_DIRECT_WIDE=1/0 forces a choice).
DirectConst direct_const(const MeshDev& m, const Batch& b, int lanes, const Ctx& c, bool mixed,
                         double tol, int max_sweeps) {
  const int n_sm = c.n_sm;
  DirectConst kc;
  memset(&kc, 0, sizeof(kc));
  kc.rowptr = m.rowptr.as<int32_t>();
  kc.colidx = m.colidx.as<int32_t>();
  kc.iperm = m.iperm.as<int32_t>();
  kc.perm = m.perm.as<int32_t>();
  kc.M = b.Mv.as<double>();
  kc.K = b.qoi_kind == MQS_QOI_ENERGY ? b.Kv.as<double>() : nullptr;
  kc.vs = b.n;
  kc.F = m.F.as<double>();
  kc.n = m.n_free;
  kc.bw = m.bw;
  kc.n_phases = m.n_phases;
  kc.qoi_kind = b.qoi_kind;
  kc.omega = kTwoPi * b.freq;
  const int forced = env_int("MQS_DIRECT_WIDE", -1);
  const bool wide = forced >= 0 ? forced == 1 : lanes < 2 * n_sm;
  kc.w_in_smem = (wide && m.n_free <= direct_smem_max_n(mixed ? 1 : 0)) ? 1 : 0;
  kc.mixed = mixed ? 1 : 0;
  kc.tol2 = tol * tol;
  kc.max_sweeps = max_sweeps;
  kc.cluster = direct_cluster(m, lanes, n_sm, mixed, wide);
  kc.stall_test = c.test_hook == MQS_TEST_HOOK_STALL ? 1 : 0;
  return kc;
}

DirectLane direct_lane(const MeshDev& m, const Batch& b, const FactorSet& f, int sample,
                       double* a0, double* a1, double* y, double* w, double* rhs,
                       double* qoi_out, int32_t* status_out, int n_steps, int64_t k0,
                       int init_from_a0) {
  DirectLane d;
  memset(&d, 0, sizeof(d));
  const size_t fstride = (size_t)m.n_free * (m.bw + 1);
  d.LB = f.LB.as<double>() + fstride * sample;
  d.invd = f.invd.as<double>() + (size_t)m.n_free * sample;
  d.Binv = f.Binv.as<double>() + (size_t)block_count(m.n_free) * 32 * 32 * sample;
  const size_t bo = cluster_bstride(m) * sample;
  d.B64 = f.B64.as<double>() + bo;
  d.B64T = f.B64T.as<double>() + bo;
  d.C1 = f.C1.as<double>() + bo;
  d.C2 = f.C2.as<double>() + bo;
  d.D1 = f.D1.as<double>() + bo;
  d.D2 = f.D2.as<double>() + bo;
  d.LBf = f.LBf.as<float>() + fstride * sample;
  d.invdf = f.invdf.as<float>() + (size_t)m.n_free * sample;
  d.Binvf = f.Binvf.as<float>() + (size_t)block_count(m.n_free) * 32 * 32 * sample;
  for (auto& v : b.vsets)
    if (v->dt == f.dt) d.Av = v->A.as<double>() + sample;
  d.b = rhs;
  d.status_out = status_out;
  d.a0 = a0;
  d.a1 = a1;
  d.y = y;
  d.w = w;
  d.qoi_out = qoi_out;
  d.vcol = sample;
  d.qoi_scale = 1.0;
  const int R = m.n_regions, P = m.n_phases;
  const double* p = b.hparams.data() + (size_t)sample * b.n_params;
  for (int q = 0; q < kMaxPhases; ++q) {
    d.amp[q] = q < P ? p[2 * R] * p[2 * R + 1 + q] : 0.0;
    d.phase[q] = q < P ? p[2 * R + 1 + P + q] : 0.0;
  }
  d.dt = f.dt;
  d.t0 = b.t0;
  d.k0 = k0;
  d.n_steps = n_steps;
  d.init_from_a0 = init_from_a0;
  d.sample = sample;
  return d;
}

int upload_direct(mqs_ctx* ctx, DirectSet& ds) {
  MQS_TRY(ds.desc.ensure(std::max<size_t>(1, ds.host.size()) * sizeof(DirectLane)));
  if (!ds.host.empty())
    MQS_CUDA_TRY(cudaMemcpyAsync(ds.desc.p, ds.host.data(), ds.host.size() * sizeof(DirectLane),
                                 cudaMemcpyHostToDevice, ctx->c.stream));
  return MQS_OK;
}

// Sequential stepping with the banded solver: lanes [0, nf) level l, [nf, nf+nc) level l-1.
int run_plain_direct(mqs_ctx* ctx, Batch& b, const MeshDev& m, FactorSet* ff, int nsf,
                     FactorSet* fc, int nsc, bool mixed, double tol, int max_sweeps) {
  const int nf = ff ? b.n : 0, nc = fc ? b.n : 0;
  DirectSet& ds = b.dplain;
  MQS_TRY(ds.ensure(nf + nc, m.n_free));
  const DirectConst kc = direct_const(m, b, nf + nc, ctx->c, mixed, tol, max_sweeps);
  if (kc.cluster) {
    if (ff) MQS_TRY(ensure_couplings(ctx, b, m, *ff));
    if (fc) MQS_TRY(ensure_couplings(ctx, b, m, *fc));
  }
  MQS_CUDA_TRY(cudaMemsetAsync(ds.qraw.p, 0, (size_t)(nf + nc) * sizeof(double), ctx->c.stream));
  MQS_CUDA_TRY(cudaMemsetAsync(ds.status.p, 0, (size_t)(nf + nc) * sizeof(int32_t), ctx->c.stream));
  ds.host.clear();
  for (int s = 0; s < nf; ++s)
    ds.host.push_back(direct_lane(m, b, *ff, s, ds.v(s, 0), ds.v(s, 1), ds.v(s, 2), ds.v(s, 3),
                                  ds.v(s, 4), ds.qraw.as<double>() + s,
                                  ds.status.as<int32_t>() + s, nsf, 0, 0));
  for (int s = 0; s < nc; ++s) {
    const int l = nf + s;
    ds.host.push_back(direct_lane(m, b, *fc, s, ds.v(l, 0), ds.v(l, 1), ds.v(l, 2), ds.v(l, 3),
                                  ds.v(l, 4), ds.qraw.as<double>() + l,
                                  ds.status.as<int32_t>() + l, nsc, 0, 0));
  }
  b.nf_direct = nf;
  MQS_TRY(upload_direct(ctx, ds));
  MQS_TRY(prof_mark(ctx->c, 0, true));
  if (kc.cluster)
    MQS_TRY(launch_cluster(ds.desc.as<DirectLane>(), nf + nc, kc, ctx->c.stream));
  else
    MQS_TRY(launch_direct(ds.desc.as<DirectLane>(), nf + nc, kc, ctx->c.stream));
  MQS_TRY(prof_mark(ctx->c, 0, false));
  b.stats[1] += (double)nf * nsf + (double)nc * nsc;
  b.stats[2] += (double)nf * nsf + (double)nc * nsc;
  b.stats[6] += (double)nf * nsf + (double)nc * nsc;
  return MQS_OK;
}

int run_parareal_pipelined(mqs_ctx* ctx, Batch& b, const MeshDev& m, FactorSet& fF,
                           FactorSet& fC, int n_steps, int M, int max_iters, double tol,
                           int& iters_out, cudaEvent_t fine_ready, const DirectConst& kc_in,
                           const DirectConst& kchain_in);

// fine_ready: event after which fF is complete (the fine factorisation ran on
// the side stream), waited for before the first fine batch; null if fF is
// already ordered on the main stream.
int run_parareal_direct(mqs_ctx* ctx, Batch& b, const MeshDev& m, FactorSet& fF,
                        FactorSet& fC, int n_steps, int M, int cf, int max_iters, double tol,
                        bool mixed, double ir_tol, int max_sweeps, int& iters_out,
                        cudaEvent_t fine_ready) {
  const cudaStream_t st = ctx->c.stream;
  const int S = n_steps / M, Sc = S / cf, ns = b.n, n = m.n_free;
  const int lanes = ns * M;
  const size_t field = (size_t)lanes * n * sizeof(double);
  MQS_TRY(b.U.ensure(field));
  MQS_TRY(b.G.ensure(field));
  MQS_TRY(b.E.ensure(field));
  MQS_TRY(b.jump2.ensure((size_t)lanes * sizeof(double)));
  MQS_TRY(b.norm2.ensure((size_t)lanes * sizeof(double)));
  MQS_TRY(b.dpar.ensure(lanes, n));
  MQS_TRY(b.dchain.ensure(ns, n));
  MQS_CUDA_TRY(cudaMemsetAsync(b.U.p, 0, field, st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.G.p, 0, field, st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.norm2.p, 0, (size_t)lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.dpar.qraw.p, 0, (size_t)lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.dpar.status.p, 0, (size_t)lanes * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.dchain.status.p, 0, (size_t)ns * sizeof(int32_t), st));
  const DirectConst kc = direct_const(m, b, lanes, ctx->c, mixed, ir_tol, max_sweeps);
  DirectConst kchain = direct_const(m, b, ns, ctx->c, mixed, ir_tol, max_sweeps);
  {   // env MQS_CHAIN_CLUSTER=1/2/4/8 forces the coarse sweep's cluster size
    const int fc = env_int("MQS_CHAIN_CLUSTER", 0);
    if (kchain.cluster && (fc == 1 || fc == 2 || fc == 4 || fc == 8)) kchain.cluster = fc;
  }
  if (kc.cluster && !fine_ready) MQS_TRY(ensure_couplings(ctx, b, m, fF));
  if (kchain.cluster) MQS_TRY(ensure_couplings(ctx, b, m, fC));
  if (kc.cluster && kchain.cluster && env_int("MQS_PARAREAL_PIPELINE", 1) != 0)
    return run_parareal_pipelined(ctx, b, m, fF, fC, n_steps, M, max_iters, tol, iters_out,
                                  fine_ready, kc, kchain);
  auto fine = [&](const DirectSet& d, int nl) -> int {
    return kc.cluster ? launch_cluster(d.desc.as<DirectLane>(), nl, kc, st)
                      : launch_direct(d.desc.as<DirectLane>(), nl, kc, st);
  };
  auto chain = [&](const DirectChain& c) -> int {
    return kchain.cluster ? launch_cluster_chain(b.dchain.desc.as<DirectLane>(), ns, kchain, c, st)
                          : launch_direct_chain(b.dchain.desc.as<DirectLane>(), ns, kchain, c, st);
  };
  DirectSet& dc = b.dchain;
  dc.host.clear();
  for (int s = 0; s < ns; ++s)
    dc.host.push_back(direct_lane(m, b, fC, s, dc.v(s, 0), dc.v(s, 1), dc.v(s, 2), dc.v(s, 3),
                                  dc.v(s, 4), dc.qraw.as<double>() + s,
                                  dc.status.as<int32_t>() + s, Sc, 0, 1));
  MQS_TRY(upload_direct(ctx, dc));
  DirectChain ch;
  ch.U_prev = ch.U_cur = b.U.as<double>();
  ch.E = b.E.as<double>();
  ch.G = b.G.as<double>();
  ch.M = M;
  ch.steps_per_slice = Sc;
  ch.jump2 = b.jump2.as<double>();
  ch.norm2 = b.norm2.as<double>();
  ch.s_first = ch.s_begin = 0;
  ch.s_end = M;
  ch.first_sweep = 1;
  MQS_CUDA_TRY(cudaMemsetAsync(b.jump2.p, 0, (size_t)lanes * sizeof(double), st));
  MQS_TRY(prof_mark(ctx->c, 1, true));
  MQS_TRY(chain(ch));
  MQS_TRY(prof_mark(ctx->c, 1, false));
  double exec_steps = (double)ns * (M - 1) * Sc, chain_steps = exec_steps, fine_steps = 0.0;
  std::vector<double> hj((size_t)lanes), hn((size_t)lanes);
  DirectSet& dp = b.dpar;
  int k = 0;
  for (k = 1; k <= max_iters; ++k) {
    MQS_CUDA_TRY(cudaMemcpyAsync(b.E.p, b.U.p, field, cudaMemcpyDeviceToDevice, st));
    dp.host.clear();
    for (int s = 0; s < ns; ++s)
      for (int j = k - 1; j < M; ++j) {
        const int l = s * M + j, c = (int)dp.host.size();
        dp.host.push_back(direct_lane(m, b, fF, s, b.E.as<double>() + (size_t)l * n, dp.v(c, 1),
                                      dp.v(c, 2), dp.v(c, 3), dp.v(c, 4),
                                      dp.qraw.as<double>() + l, dp.status.as<int32_t>() + l, S,
                                      (int64_t)j * S, 1));
      }
    fine_steps += (double)dp.host.size() * S;
    exec_steps += (double)dp.host.size() * S;
    if (k == 1 && fine_ready) MQS_CUDA_TRY(cudaStreamWaitEvent(st, fine_ready, 0));
    MQS_TRY(upload_direct(ctx, dp));
    MQS_TRY(prof_mark(ctx->c, 0, true));
    MQS_TRY(fine(dp, (int)dp.host.size()));
    MQS_TRY(prof_mark(ctx->c, 0, false));
    MQS_CUDA_TRY(cudaMemsetAsync(b.jump2.p, 0, (size_t)lanes * sizeof(double), st));
    if (k - 1 <= M - 2) {
      ch.s_first = ch.s_begin = k - 1;
      ch.first_sweep = 0;
      MQS_TRY(prof_mark(ctx->c, 1, true));
      MQS_TRY(chain(ch));
      MQS_TRY(prof_mark(ctx->c, 1, false));
      exec_steps += (double)ns * (M - 1 - (k - 1)) * Sc;
      chain_steps += (double)ns * (M - 1 - (k - 1)) * Sc;
    }
    MQS_CUDA_TRY(cudaMemcpyAsync(hj.data(), b.jump2.p, hj.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    MQS_CUDA_TRY(cudaMemcpyAsync(hn.data(), b.norm2.p, hn.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    MQS_CUDA_TRY(cudaStreamSynchronize(st));
    bool all = true;
    for (int s = 0; s < ns; ++s) {
      double num = 0.0, den = 0.0;
      for (int j = 0; j < M; ++j) {
        num = std::max(num, std::sqrt(hj[(size_t)s * M + j]));
        den = std::max(den, std::sqrt(hn[(size_t)s * M + j]));
      }
      const double jump = den > 0.0 ? num / den : num;
      if (!(jump <= tol)) all = false;
    }
    if (all || k >= M) break;
  }
  iters_out = std::min(k, max_iters);
  b.E_final = b.E.as<double>();
  b.stats[1] += exec_steps;
  b.stats[2] += (double)ns * n_steps;
  b.stats[6] += fine_steps;
  b.stats[7] += chain_steps;
  return MQS_OK;
}

// Parareal with the coarse sweep and the fine propagation overlapped (the
// same arithmetic as run_parareal_direct, so bitwise the same results).  The
// slices are cut into J chunks of c slices.  Iteration k's fine chunk j needs
// only the slice starts that iteration k - 1's sweep wrote up to the end of
// chunk j, and the sweep of chunk j needs only that chunk's fine ends, so
//   fine(k, j)  waits for  sweep(k - 1, j)          (one stream per chunk)
//   sweep(k, j) waits for  fine(k, j), sweep(k, j - 1)   (the main stream)
// and the sweep of one chunk runs while later chunks still propagate.  Slice
// starts and fine ends are double-buffered by iteration parity (U_k, E_k,
// per-slice QoI partials), so iteration k + 1 can be enqueued before the host
// knows whether iteration k met the stopping rule; per-iteration jump and norm
// squares go to host-mapped memory, read once the last sweep chunk of
// iteration k has run.  When iteration K stops, the host raises the
// cancellation word (host-mapped) and the kernels of iteration K + 1 leave at
// their next step boundary; the call drains them before it returns.
// Cluster stepping kernels only (they carry the cancellation check).
int run_parareal_pipelined(mqs_ctx* ctx, Batch& b, const MeshDev& m, FactorSet& fF,
                           FactorSet& fC, int n_steps, int M, int max_iters, double tol,
                           int& iters_out, cudaEvent_t fine_ready, const DirectConst& kc_in,
                           const DirectConst& kchain_in) {
  Ctx& c = ctx->c;
  const cudaStream_t st = c.stream;
  const int S = n_steps / M, Sc = S / (int)std::lround(fC.dt / fF.dt), ns = b.n, n = m.n_free;
  const int lanes = ns * M;
  const int64_t field = (int64_t)lanes * n;
  const int cs = std::max(1, M / 16);              // slices per chunk
  const int J = (M + cs - 1) / cs;                 // chunks
  MQS_TRY(ensure_pipeline(c, J));
  MQS_TRY(b.U.ensure(2 * field * sizeof(double)));
  MQS_TRY(b.E.ensure(2 * field * sizeof(double)));
  MQS_TRY(b.G.ensure(field * sizeof(double)));
  MQS_TRY(b.qraw2.ensure(2 * (size_t)lanes * sizeof(double)));
  MQS_TRY(b.pdesc.ensure(2 * (size_t)lanes * sizeof(DirectLane)));
  MQS_TRY(b.dpar.ensure(lanes, n));
  MQS_TRY(b.dchain.ensure(ns, n));
  const size_t hist = (size_t)(max_iters + 2) * lanes * sizeof(double);
  MQS_TRY(b.jhist.ensure(hist));
  MQS_TRY(b.nhist.ensure(hist));
  MQS_TRY(b.stop.ensure(sizeof(int32_t)));
  // nothing of an earlier call touches the mapped words any more: every
  // pipelined call drains its cancelled kernels before it returns
  memset(b.jhist.h, 0, hist);
  memset(b.nhist.h, 0, hist);
  volatile int32_t* stop_h = static_cast<volatile int32_t*>(b.stop.h);
  *stop_h = INT32_MAX;
  double* U0 = b.U.as<double>();
  double* E0 = b.E.as<double>();
  double* q2 = b.qraw2.as<double>();
  MQS_CUDA_TRY(cudaMemsetAsync(U0, 0, 2 * field * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(q2, 0, 2 * (size_t)lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.dpar.status.p, 0, (size_t)lanes * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(b.dchain.status.p, 0, (size_t)ns * sizeof(int32_t), st));
  DirectConst kc = kc_in, kchain = kchain_in;
  kc.stop = kchain.stop = static_cast<const volatile int32_t*>(b.stop.d);
  // fine-lane descriptors of both parities, slice-major (chunk = contiguous range)
  std::vector<DirectLane> pd((size_t)2 * lanes);
  for (int par = 0; par < 2; ++par)
    for (int j = 0; j < M; ++j)
      for (int smp = 0; smp < ns; ++smp) {
        const int l = smp * M + j;
        DirectLane d = direct_lane(m, b, fF, smp, E0 + par * field + (int64_t)l * n,
                                   b.dpar.v(l, 1), b.dpar.v(l, 2), b.dpar.v(l, 3),
                                   b.dpar.v(l, 4), q2 + (size_t)par * lanes + l,
                                   b.dpar.status.as<int32_t>() + l, S, (int64_t)j * S, 1);
        d.a_init = U0 + (par ^ 1) * field + (int64_t)l * n;   // U of iteration k - 1
        pd[(size_t)par * lanes + (size_t)j * ns + smp] = d;
      }
  MQS_CUDA_TRY(cudaMemcpyAsync(b.pdesc.p, pd.data(), pd.size() * sizeof(DirectLane),
                               cudaMemcpyHostToDevice, st));
  DirectSet& dc = b.dchain;
  dc.host.clear();
  for (int smp = 0; smp < ns; ++smp)
    dc.host.push_back(direct_lane(m, b, fC, smp, dc.v(smp, 0), dc.v(smp, 1), dc.v(smp, 2),
                                  dc.v(smp, 3), dc.v(smp, 4), dc.qraw.as<double>() + smp,
                                  dc.status.as<int32_t>() + smp, Sc, 0, 1));
  MQS_TRY(upload_direct(ctx, dc));
  // the fine chunk streams start after everything enqueued so far
  MQS_CUDA_TRY(cudaEventRecord(c.ev_fork, st));
  for (int j = 0; j < J; ++j) MQS_CUDA_TRY(cudaStreamWaitEvent(c.fine_st[j], c.ev_fork, 0));
  if (fine_ready)
    for (int j = 0; j < J; ++j) MQS_CUDA_TRY(cudaStreamWaitEvent(c.fine_st[j], fine_ready, 0));
  const DirectLane* dpd = b.pdesc.as<DirectLane>();
  double* jh = static_cast<double*>(b.jhist.d);
  double* nh = static_cast<double*>(b.nhist.d);
  double exec_steps = 0.0, chain_steps = 0.0, fine_steps = 0.0;
  // sweep of iteration k (k = 0: the initial coarse sweep), chunk by chunk
  auto sweep = [&](int k) -> int {
    const int pk = k & 1;
    DirectChain ch;
    ch.U_prev = U0 + (pk ^ 1) * field;
    ch.U_cur = U0 + pk * field;
    ch.E = E0 + pk * field;
    ch.G = b.G.as<double>();
    ch.M = M;
    ch.steps_per_slice = Sc;
    ch.jump2 = jh + (size_t)k * lanes;
    ch.norm2 = nh + (size_t)k * lanes;
    ch.s_first = k == 0 ? 0 : k - 1;
    ch.first_sweep = k == 0 ? 1 : 0;
    DirectConst kk = kchain;
    kk.iter = k;
    for (int j = 0; j < J; ++j) {
      const int lo = std::max(j * cs, ch.s_first), hi = std::min((j + 1) * cs, M - 1);
      if (k > 0) MQS_CUDA_TRY(cudaStreamWaitEvent(st, c.ev_fine[pk][j], 0));
      if (lo < hi) {
        ch.s_begin = lo;
        ch.s_end = hi;
        MQS_TRY(prof_mark(c, 1, true));
        MQS_TRY(launch_cluster_chain(dc.desc.as<DirectLane>(), ns, kk, ch, st));
        MQS_TRY(prof_mark(c, 1, false));
      }
      MQS_CUDA_TRY(cudaEventRecord(c.ev_sweep[pk][j], st));
    }
    return MQS_OK;
  };
  // fine propagation of iteration k >= 1 on slices k - 1 .. M - 1, chunk by chunk
  auto fine = [&](int k) -> int {
    const int pk = k & 1;
    DirectConst kk = kc;
    kk.iter = k;
    for (int j = 0; j < J; ++j) {
      const int lo = std::max(j * cs, k - 1), hi = std::min((j + 1) * cs, M);
      const cudaStream_t fs = c.fine_st[j];
      MQS_CUDA_TRY(cudaStreamWaitEvent(fs, c.ev_sweep[pk ^ 1][j], 0));
      if (lo < hi) {
        MQS_TRY(prof_mark(c, 0, true, fs));
        MQS_TRY(launch_cluster(dpd + (size_t)pk * lanes + (size_t)lo * ns, (hi - lo) * ns, kk,
                               fs));
        MQS_TRY(prof_mark(c, 0, false, fs));
      }
      MQS_CUDA_TRY(cudaEventRecord(c.ev_fine[pk][j], fs));
    }
    return MQS_OK;
  };
  MQS_TRY(sweep(0));
  int K = 0;
  auto enqueue = [&](int k) -> int {
    MQS_TRY(fine(k));
    return sweep(k);
  };
  MQS_TRY(enqueue(1));
  for (int k = 1; k <= max_iters; ++k) {
    if (k + 1 <= max_iters && k < M) MQS_TRY(enqueue(k + 1));   // ahead, speculatively
    MQS_CUDA_TRY(cudaEventSynchronize(c.ev_sweep[k & 1][J - 1]));
    const double* hj = static_cast<const double*>(b.jhist.h) + (size_t)k * lanes;
    bool all = true;
    for (int smp = 0; smp < ns; ++smp) {
      double num = 0.0, den = 0.0;
      for (int j = 0; j < M; ++j) {
        // the last iteration <= k that wrote slice start j is min(k, j)
        const double* hn = static_cast<const double*>(b.nhist.h) + (size_t)std::min(k, j) * lanes;
        num = std::max(num, std::sqrt(hj[(size_t)smp * M + j]));
        den = std::max(den, std::sqrt(hn[(size_t)smp * M + j]));
      }
      const double jump = den > 0.0 ? num / den : num;
      if (!(jump <= tol)) all = false;
    }
    K = k;
    fine_steps += (double)ns * (M - (k - 1)) * S;
    if (all || k >= M || k >= max_iters) break;
  }
  // cancel the iteration enqueued ahead (if any) and drain it
  *stop_h = K;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  for (int j = 0; j < J; ++j) {
    MQS_CUDA_TRY(cudaEventRecord(c.ev_fjoin[j], c.fine_st[j]));
    MQS_CUDA_TRY(cudaStreamWaitEvent(st, c.ev_fjoin[j], 0));
  }
  MQS_TRY(gather_parareal_qraw(q2, lanes, M, K, b.dpar.qraw.as<double>(), st));
  MQS_CUDA_TRY(cudaStreamSynchronize(st));
  iters_out = K;
  b.E_final = E0 + (K & 1) * field;
  // sweeps of iterations 0..K (those of K + 1, enqueued ahead, were cancelled)
  for (int k = 0; k <= K; ++k) chain_steps += (double)ns * (M - 1 - std::max(0, k - 1)) * Sc;
  exec_steps = fine_steps + chain_steps;
  b.stats[1] += exec_steps;
  b.stats[2] += (double)ns * n_steps;
  b.stats[6] += fine_steps;
  b.stats[7] += chain_steps;
  return MQS_OK;
}

}  // namespace

extern "C" {

const char* mqs_last_error(void) { return g_err.c_str(); }

int mqs_create(mqs_ctx** out, int device, void* cuda_stream) {
  clear_error();
  if (!out) {
    set_error("null output pointer");
    return MQS_EINVAL;
  }
  int count = 0;
  MQS_CUDA_TRY(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    set_error("device %d out of range (%d devices)", device, count);
    return MQS_EINVAL;
  }
  MQS_CUDA_TRY(cudaSetDevice(device));
  int major = 0;
  MQS_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
  if (major < 9) {
    set_error("device %d has compute capability %d.x; thread-block clusters need >= 9.0",
              device, major);
    return MQS_EINVAL;
  }
  auto* ctx = new (std::nothrow) mqs_ctx();
  if (!ctx) {
    set_error("out of host memory");
    return MQS_ENOMEM;
  }
  ctx->c.device = device;
  ctx->c.stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&ctx->c.n_sm, cudaDevAttrMultiProcessorCount, device);
  *out = ctx;
  return MQS_OK;
}

int mqs_set_stream(mqs_ctx* ctx, void* cuda_stream) {
  MQS_TRY(enter(ctx));
  ctx->c.stream = static_cast<cudaStream_t>(cuda_stream);
  return MQS_OK;
}

int mqs_destroy(mqs_ctx* ctx) {
  if (!ctx) return MQS_OK;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  delete ctx;
  return MQS_OK;
}

int mqs_upload_mesh(mqs_ctx* ctx, int32_t n_nodes, const double* xy, int32_t n_tri,
                    const int32_t* tri, const int32_t* region, int32_t n_regions,
                    const uint8_t* dirichlet, const int32_t* src_phase, const double* src_coef,
                    int32_t n_phases, int32_t* mesh_id) {
  MQS_TRY(enter(ctx));
  if (!xy || !tri || !region || !dirichlet || !src_phase || !src_coef || !mesh_id) {
    set_error("null array argument");
    return MQS_EINVAL;
  }
  if (n_nodes < 3 || n_tri < 1 || n_regions < 1 || n_regions > kMaxRegions || n_phases < 0 ||
      n_phases > kMaxPhases || (int64_t)n_tri * 9 >= (int64_t)INT32_MAX) {
    set_error("bad mesh sizes: nodes %d, triangles %d, regions %d, phases %d", n_nodes, n_tri,
              n_regions, n_phases);
    return MQS_EINVAL;
  }
  for (int64_t e = 0; e < n_tri; ++e) {
    for (int v = 0; v < 3; ++v)
      if (tri[3 * e + v] < 0 || tri[3 * e + v] >= n_nodes) {
        set_error("triangle %lld has node id %d out of range", (long long)e, tri[3 * e + v]);
        return MQS_EINVAL;
      }
    if (region[e] < 0 || region[e] >= n_regions) {
      set_error("triangle %lld has region %d out of range", (long long)e, region[e]);
      return MQS_EINVAL;
    }
    if (src_phase[e] < -1 || src_phase[e] >= n_phases) {
      set_error("triangle %lld has source phase %d out of range", (long long)e, src_phase[e]);
      return MQS_EINVAL;
    }
    const double* p0 = xy + 2 * (int64_t)tri[3 * e];
    const double* p1 = xy + 2 * (int64_t)tri[3 * e + 1];
    const double* p2 = xy + 2 * (int64_t)tri[3 * e + 2];
    const double d = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]);
    if (!(std::fabs(d) > 0.0) || !std::isfinite(d)) {
      set_error("triangle %lld is degenerate", (long long)e);
      return MQS_EINVAL;
    }
  }
  auto mesh = std::unique_ptr<MeshDev>(new MeshDev());
  MeshDev& m = *mesh;
  m.n_nodes = n_nodes;
  m.n_tri = n_tri;
  m.n_regions = n_regions;
  m.n_phases = n_phases;
  std::vector<int32_t> fid(n_nodes, -1);
  for (int32_t v = 0; v < n_nodes; ++v)
    if (!dirichlet[v]) {
      fid[v] = (int32_t)m.free_node.size();
      m.free_node.push_back(v);
    }
  m.n_free = (int32_t)m.free_node.size();
  if (m.n_free == 0) {
    set_error("mesh has no free node");
    return MQS_EINVAL;
  }
  // CSR pattern over free unknowns: couplings through shared triangles
  std::vector<std::vector<int32_t>> nbr(m.n_free);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      const int32_t fa = fid[tri[3 * e + a]];
      if (fa < 0) continue;
      for (int bb = 0; bb < 3; ++bb) {
        const int32_t fb = fid[tri[3 * e + bb]];
        if (fb >= 0) nbr[fa].push_back(fb);
      }
    }
  std::vector<int32_t> rowptr(m.n_free + 1, 0), colidx, diag(m.n_free);
  for (int32_t i = 0; i < m.n_free; ++i) {
    auto& v = nbr[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    if ((int)v.size() > kMaxRowNnz) {
      set_error("free node %d has %zu couplings (limit %d)", m.free_node[i], v.size(), kMaxRowNnz);
      return MQS_EINVAL;
    }
    m.max_row_nnz = std::max<int32_t>(m.max_row_nnz, (int32_t)v.size());
    rowptr[i + 1] = rowptr[i] + (int32_t)v.size();
    diag[i] = rowptr[i] + (int32_t)(std::lower_bound(v.begin(), v.end(), i) - v.begin());
    colidx.insert(colidx.end(), v.begin(), v.end());
  }
  m.nnz = (int64_t)colidx.size();
  // reverse Cuthill-McKee ordering and the lower-band position of each nonzero
  std::vector<int32_t> perm, iperm(m.n_free), band_idx(m.nnz);
  int32_t bw = 0;
  std::vector<char> boundary(m.n_free, 0);   // free nodes sharing a triangle with a Dirichlet node
  for (int64_t e = 0; e < n_tri; ++e) {
    bool has_dir = false;
    for (int a = 0; a < 3; ++a) has_dir |= fid[tri[3 * e + a]] < 0;
    if (has_dir)
      for (int a = 0; a < 3; ++a)
        if (fid[tri[3 * e + a]] >= 0) boundary[fid[tri[3 * e + a]]] = 1;
  }
  rcm_order(m.n_free, rowptr, colidx, boundary, perm, bw);
  for (int32_t i = 0; i < m.n_free; ++i) iperm[perm[i]] = i;
  if ((int64_t)m.n_free * (bw + 1) >= (int64_t)INT32_MAX) bw = -1;   // too wide for the band solver
  for (int32_t i = 0; i < m.n_free; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t pi = iperm[i], pj = iperm[colidx[k]];
      band_idx[k] = (bw >= 0 && pj <= pi) ? pi * (bw + 1) + (pj - pi + bw) : -1;
    }
  m.bw = bw;
  // element contributions per nonzero, sorted by (nonzero, code)
  std::vector<std::pair<int32_t, int32_t>> kc;
  kc.reserve((size_t)n_tri * 9);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      const int32_t fa = fid[tri[3 * e + a]];
      if (fa < 0) continue;
      for (int bb = 0; bb < 3; ++bb) {
        const int32_t fb = fid[tri[3 * e + bb]];
        if (fb < 0) continue;
        const int32_t* beg = colidx.data() + rowptr[fa];
        const int32_t* end = colidx.data() + rowptr[fa + 1];
        const int32_t k = (int32_t)(std::lower_bound(beg, end, fb) - colidx.data());
        kc.emplace_back(k, (int32_t)(e * 9 + a * 3 + bb));
      }
    }
  std::sort(kc.begin(), kc.end());
  std::vector<int32_t> cptr(m.nnz + 1, 0), contrib(kc.size());
  for (size_t j = 0; j < kc.size(); ++j) {
    cptr[kc[j].first + 1]++;
    contrib[j] = kc[j].second;
  }
  for (int64_t k = 0; k < m.nnz; ++k) cptr[k + 1] += cptr[k];
  // source triangles per free row, sorted by (row, triangle)
  std::vector<std::pair<int32_t, int32_t>> rl;
  for (int64_t e = 0; e < n_tri; ++e) {
    if (src_phase[e] < 0) continue;
    for (int a = 0; a < 3; ++a) {
      const int32_t fa = fid[tri[3 * e + a]];
      if (fa >= 0) rl.emplace_back(fa, (int32_t)e);
    }
  }
  std::sort(rl.begin(), rl.end());
  std::vector<int32_t> lptr(m.n_free + 1, 0), load(rl.size());
  for (size_t j = 0; j < rl.size(); ++j) {
    lptr[rl[j].first + 1]++;
    load[j] = rl[j].second;
  }
  for (int32_t i = 0; i < m.n_free; ++i) lptr[i + 1] += lptr[i];
  const cudaStream_t st = ctx->c.stream;
  MQS_TRY(m.rowptr.ensure(rowptr.size() * sizeof(int32_t)));
  MQS_TRY(m.colidx.ensure(colidx.size() * sizeof(int32_t)));
  MQS_TRY(m.diag.ensure(diag.size() * sizeof(int32_t)));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.rowptr.p, rowptr.data(), rowptr.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.colidx.p, colidx.data(), colidx.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.diag.p, diag.data(), diag.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_TRY(m.perm.ensure(perm.size() * sizeof(int32_t)));
  MQS_TRY(m.iperm.ensure(iperm.size() * sizeof(int32_t)));
  MQS_TRY(m.band_idx.ensure(band_idx.size() * sizeof(int32_t)));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.perm.p, perm.data(), perm.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.iperm.p, iperm.data(), iperm.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(m.band_idx.p, band_idx.data(), band_idx.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  MQS_TRY(assemble_region_matrices(m, xy, tri, region, src_phase, src_coef, cptr, contrib, lptr,
                                   load, st));
  ctx->c.meshes.push_back(std::move(mesh));
  *mesh_id = (int32_t)ctx->c.meshes.size() - 1;
  return MQS_OK;
}

int mqs_set_solver(mqs_ctx* ctx, int32_t batch_id, int32_t solver) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (solver != MQS_SOLVER_PCG && solver != MQS_SOLVER_BANDED) {
    set_error("unknown solver %d", solver);
    return MQS_EINVAL;
  }
  b->solver = solver;
  return MQS_OK;
}

int mqs_mesh_bandwidth(mqs_ctx* ctx, int32_t mesh_id, int32_t* bandwidth) {
  MQS_TRY(enter(ctx));
  MeshDev* m = get_mesh(ctx, mesh_id);
  if (!m || !bandwidth) return MQS_EINVAL;
  *bandwidth = m->bw;
  return MQS_OK;
}

int mqs_mesh_info(mqs_ctx* ctx, int32_t mesh_id, int32_t* n_free, int64_t* nnz) {
  MQS_TRY(enter(ctx));
  MeshDev* m = get_mesh(ctx, mesh_id);
  if (!m) return MQS_EINVAL;
  if (n_free) *n_free = m->n_free;
  if (nnz) *nnz = m->nnz;
  return MQS_OK;
}

int mqs_set_samples(mqs_ctx* ctx, int32_t mesh_id, int32_t n_samples, int32_t n_params,
                    const double* params, int32_t* batch_id) {
  MQS_TRY(enter(ctx));
  MeshDev* m = get_mesh(ctx, mesh_id);
  if (!m) return MQS_EINVAL;
  if (!params || !batch_id || n_samples < 1) {
    set_error("need n_samples >= 1, params and batch_id");
    return MQS_EINVAL;
  }
  const int expect = 2 * m->n_regions + 1 + 2 * m->n_phases;
  if (n_params != expect) {
    set_error("n_params = %d, the mesh needs 2R + 1 + 2P = %d", n_params, expect);
    return MQS_EINVAL;
  }
  auto b = std::unique_ptr<Batch>(new Batch());
  b->mesh_id = mesh_id;
  b->n = n_samples;
  b->n_params = n_params;
  const size_t bytes = (size_t)n_samples * n_params * sizeof(double);
  MQS_TRY(b->params.ensure(bytes));
  MQS_CUDA_TRY(cudaMemcpyAsync(b->params.p, params, bytes, cudaMemcpyDefault, ctx->c.stream));
  b->hparams.resize((size_t)n_samples * n_params);
  MQS_CUDA_TRY(cudaMemcpyAsync(b->hparams.data(), b->params.p, bytes, cudaMemcpyDeviceToHost,
                               ctx->c.stream));
  MQS_TRY(b->qoi.ensure((size_t)n_samples * 2 * sizeof(double)));
  MQS_TRY(b->status.ensure((size_t)n_samples * sizeof(int32_t)));
  MQS_CUDA_TRY(cudaMemsetAsync(b->qoi.p, 0, (size_t)n_samples * 2 * sizeof(double), ctx->c.stream));
  MQS_CUDA_TRY(cudaMemsetAsync(b->status.p, 0, (size_t)n_samples * sizeof(int32_t), ctx->c.stream));
  if (!is_device_ptr(params)) MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  m->live_batches++;
  ctx->c.batches.push_back(std::move(b));
  *batch_id = (int32_t)ctx->c.batches.size() - 1;
  return MQS_OK;
}

int mqs_set_time(mqs_ctx* ctx, int32_t batch_id, double t0, double t_end, double freq_hz,
                 int32_t qoi_kind) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (!(t_end > t0) || !std::isfinite(t0) || !std::isfinite(t_end) || !std::isfinite(freq_hz) ||
      (qoi_kind != MQS_QOI_ENERGY && qoi_kind != MQS_QOI_JOULE)) {
    set_error("bad time window [%g, %g], frequency %g or QoI kind %d", t0, t_end, freq_hz,
              qoi_kind);
    return MQS_EINVAL;
  }
  b->t0 = t0;
  b->t_end = t_end;
  b->freq = freq_hz;
  b->qoi_kind = qoi_kind;
  b->time_set = true;
  return MQS_OK;
}

int mqs_propagate(mqs_ctx* ctx, int32_t batch_id, int32_t level, double dt_level, double dt_prev,
                  int32_t n_slices, int32_t coarse_factor, int32_t max_par_iters, double par_tol,
                  int32_t precision, double cg_tol, int32_t cg_max_iters, int32_t* par_iters_out) {
  MQS_TRY(enter(ctx));
  Batch* bp = get_batch(ctx, batch_id);
  if (!bp) return MQS_EINVAL;
  Batch& b = *bp;
  MeshDev& m = *ctx->c.meshes[b.mesh_id];
  if (!b.time_set) {
    set_error("mqs_set_time must be called before mqs_propagate");
    return MQS_EINVAL;
  }
  if ((precision != MQS_FP64 && precision != MQS_MIXED) || cg_max_iters < 1 || !(cg_tol >= 0.0) ||
      n_slices < 1 || level < 0 || dt_prev < 0.0) {
    set_error("bad precision %d, cg_tol %g, cg_max_iters %d, n_slices %d, level %d or dt_prev %g",
              precision, cg_tol, cg_max_iters, n_slices, level, dt_prev);
    return MQS_EINVAL;
  }
  const double T = b.t_end - b.t0;
  int nsf = 0, nsc = 0;
  MQS_TRY(steps_of(T, dt_level, nsf));
  if (dt_prev > 0.0) MQS_TRY(steps_of(T, dt_prev, nsc));
  if (n_slices > 1) {
    if (coarse_factor < 1 || nsf % n_slices || (nsf / n_slices) % coarse_factor ||
        max_par_iters < 1 || max_par_iters > n_slices || !(par_tol >= 0.0)) {
      set_error("Parareal needs steps (%d) divisible by slices (%d) times coarse_factor (%d) "
                "and 1 <= max_par_iters <= slices",
                nsf, n_slices, coarse_factor);
      return MQS_EINVAL;
    }
  }
  const bool mixed = precision == MQS_MIXED;
  MQS_TRY(ensure_mk(ctx, b, m));
  int rc = MQS_OK;
  if (b.solver == MQS_SOLVER_BANDED) {
    if (m.bw < 0) {
      set_error("the banded solver needs n_free * (bw + 1) < 2^31");
      return MQS_EINVAL;
    }
    FactorSet* ff = nullptr;
    cudaEvent_t fine_ready = nullptr;
    if (n_slices > 1) {
      // the fine factor (and its block couplings) on the side stream, beside
      // the coarse factorisation and the first coarse sweep
      MQS_TRY(ensure_side(ctx->c));
      MQS_CUDA_TRY(cudaEventRecord(ctx->c.ev_fork, ctx->c.stream));
      MQS_CUDA_TRY(cudaStreamWaitEvent(ctx->c.side, ctx->c.ev_fork, 0));
      {
        OnSide on(ctx->c);
        ff = factor_set(ctx, b, m, dt_level, mixed, rc);
        if (!ff) return rc;
        const DirectConst kc = direct_const(m, b, b.n * n_slices, ctx->c, mixed, cg_tol,
                                            cg_max_iters);
        if (kc.cluster) MQS_TRY(ensure_couplings(ctx, b, m, *ff));
        MQS_CUDA_TRY(cudaEventRecord(ctx->c.ev_join, ctx->c.side));
      }
      fine_ready = ctx->c.ev_join;
    } else {
      ff = factor_set(ctx, b, m, dt_level, mixed, rc);
      if (!ff) return rc;
    }
    FactorSet* fc = nullptr;
    if (dt_prev > 0.0 && !(fc = factor_set(ctx, b, m, dt_prev, mixed, rc))) return rc;
    // a step size equal to the fine one shares the fine factor, which the side
    // stream may still be computing: the main stream waits for it first
    if (fine_ready && fc == ff) MQS_CUDA_TRY(cudaStreamWaitEvent(ctx->c.stream, fine_ready, 0));
    b.level = level;
    b.has_coarse = fc != nullptr;
    for (double& x : b.stats) x = 0.0;
    b.stats[3] = m.n_free;
    int par_iters = 0;
    const cudaStream_t st = ctx->c.stream;
    if (n_slices == 1) {
      MQS_TRY(run_plain_direct(ctx, b, m, ff, nsf, fc, nsc, mixed, cg_tol, cg_max_iters));
      b.mode = 3;
      b.M = 1;
      MQS_TRY(finish_qoi(b.dplain.qraw.as<double>(),
                         fc ? b.dplain.qraw.as<double>() + b.nf_direct : nullptr, b.n, 1,
                         qoi_scale(b.qoi_kind, nsf, dt_level),
                         fc ? qoi_scale(b.qoi_kind, nsc, dt_prev) : 0.0, b.qoi.as<double>(), st));
    } else {
      // the companion level-(l-1) solve of each sample runs on the side stream,
      // beside the Parareal iterations (its factor was formed on the main stream)
      cudaEvent_t comp_done = nullptr;
      if (fc) {
        MQS_CUDA_TRY(cudaEventRecord(ctx->c.ev_comp0, ctx->c.stream));
        MQS_CUDA_TRY(cudaStreamWaitEvent(ctx->c.side, ctx->c.ev_comp0, 0));
        {
          OnSide on(ctx->c);
          MQS_TRY(run_plain_direct(ctx, b, m, nullptr, 0, fc, nsc, mixed, cg_tol, cg_max_iters));
          MQS_CUDA_TRY(cudaEventRecord(ctx->c.ev_comp1, ctx->c.side));
        }
        comp_done = ctx->c.ev_comp1;
      }
      FactorSet* fC = factor_set(ctx, b, m, dt_level * coarse_factor, mixed, rc);
      if (!fC) return rc;
      if (fine_ready && fC == ff)   // coarse_factor 1: the coarse sweep uses the fine factor
        MQS_CUDA_TRY(cudaStreamWaitEvent(ctx->c.stream, fine_ready, 0));
      MQS_TRY(run_parareal_direct(ctx, b, m, *ff, *fC, nsf, n_slices, coarse_factor,
                                  max_par_iters, par_tol, mixed, cg_tol, cg_max_iters,
                                  par_iters, fine_ready));
      if (comp_done) MQS_CUDA_TRY(cudaStreamWaitEvent(ctx->c.stream, comp_done, 0));
      b.mode = 4;
      b.M = n_slices;
      MQS_TRY(finish_qoi(b.dpar.qraw.as<double>(), fc ? b.dplain.qraw.as<double>() : nullptr,
                         b.n, n_slices, qoi_scale(b.qoi_kind, nsf, dt_level),
                         fc ? qoi_scale(b.qoi_kind, nsc, dt_prev) : 0.0, b.qoi.as<double>(), st));
    }
    if (par_iters_out) *par_iters_out = par_iters;
    return MQS_OK;
  }
  ValueSet* vf = value_set(ctx, b, m, dt_level, mixed, rc);
  if (!vf) return rc;
  ValueSet* vc = nullptr;
  if (dt_prev > 0.0) {
    vc = value_set(ctx, b, m, dt_prev, mixed, rc);
    if (!vc) return rc;
  }
  b.level = level;
  b.has_coarse = vc != nullptr;
  for (double& s : b.stats) s = 0.0;
  b.stats[3] = m.n_free;
  const cudaStream_t st = ctx->c.stream;
  int par_iters = 0;
  if (n_slices == 1) {
    MQS_TRY(run_plain(ctx, b, m, vf, nsf, vc, nsc, precision, cg_tol, cg_max_iters));
    b.mode = 1;
    b.M = 1;
    MQS_TRY(finish_qoi(b.plain.qraw.as<double>(),
                       vc ? b.plain.qraw.as<double>() + b.nf_pad : nullptr, b.n, 1,
                       qoi_scale(b.qoi_kind, nsf, dt_level),
                       vc ? qoi_scale(b.qoi_kind, nsc, dt_prev) : 0.0, b.qoi.as<double>(), st));
    MQS_CUDA_TRY(cudaMemsetAsync(b.status.p, 0, (size_t)b.n * sizeof(int32_t), st));
  } else {
    // companion level-(l-1) solve first (sequential), then Parareal on level l
    if (vc) MQS_TRY(run_plain(ctx, b, m, nullptr, 0, vc, nsc, precision, cg_tol, cg_max_iters));
    ValueSet* vC = value_set(ctx, b, m, dt_level * coarse_factor, mixed, rc);
    if (!vC) return rc;
    MQS_TRY(run_parareal(ctx, b, m, *vf, *vC, nsf, n_slices, coarse_factor, max_par_iters,
                         par_tol, precision, cg_tol, cg_max_iters, par_iters));
    b.mode = 2;
    b.M = n_slices;
    MQS_TRY(finish_qoi(b.par.qraw.as<double>(), vc ? b.plain.qraw.as<double>() : nullptr, b.n,
                       n_slices, qoi_scale(b.qoi_kind, nsf, dt_level),
                       vc ? qoi_scale(b.qoi_kind, nsc, dt_prev) : 0.0, b.qoi.as<double>(), st));
    MQS_CUDA_TRY(cudaMemsetAsync(b.status.p, 0, (size_t)b.n * sizeof(int32_t), st));
  }
  if (par_iters_out) *par_iters_out = par_iters;
  return MQS_OK;
}

int mqs_read_qoi(mqs_ctx* ctx, int32_t batch_id, double* qoi, int32_t* status) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (!qoi) {
    set_error("null qoi array");
    return MQS_EINVAL;
  }
  const cudaStream_t st = ctx->c.stream;
  MQS_CUDA_TRY(cudaMemcpyAsync(qoi, b->qoi.p, (size_t)b->n * 2 * sizeof(double), cudaMemcpyDefault,
                               st));
  if (status) {
    // or the per-lane status bits of every solve of the sample
    std::vector<int32_t> out((size_t)b->n, 0);
    auto fold = [&](const LaneSet& ls, int lanes, int lps, int off) -> int {
      std::vector<int32_t> h((size_t)lanes);
      MQS_CUDA_TRY(cudaMemcpyAsync(h.data(), ls.status.as<int32_t>() + off, lanes * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, st));
      MQS_CUDA_TRY(cudaStreamSynchronize(st));
      for (int l = 0; l < lanes; ++l) out[l / lps] |= h[l];
      return MQS_OK;
    };
    if (b->mode == 1) {
      MQS_TRY(fold(b->plain, b->n, 1, 0));
      if (b->has_coarse) MQS_TRY(fold(b->plain, b->n, 1, b->nf_pad));
    } else if (b->mode == 2) {
      MQS_TRY(fold(b->par, b->n * b->M, b->M, 0));
      MQS_TRY(fold(b->chain, b->n, 1, 0));
      if (b->has_coarse) MQS_TRY(fold(b->plain, b->n, 1, 0));
    } else if (b->mode >= 3) {
      auto fold_direct = [&](const DirectSet& ds, int lanes, int lps, int off) -> int {
        if (lanes <= 0) return MQS_OK;
        std::vector<int32_t> hs((size_t)lanes);
        MQS_CUDA_TRY(cudaMemcpyAsync(hs.data(), ds.status.as<int32_t>() + off,
                                     lanes * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MQS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int l = 0; l < lanes; ++l) out[l / lps] |= hs[l];
        return MQS_OK;
      };
      if (b->mode == 3) {
        MQS_TRY(fold_direct(b->dplain, b->n, 1, 0));
        if (b->has_coarse) MQS_TRY(fold_direct(b->dplain, b->n, 1, b->nf_direct));
      } else {
        MQS_TRY(fold_direct(b->dpar, b->n * b->M, b->M, 0));
        MQS_TRY(fold_direct(b->dchain, b->n, 1, 0));
        if (b->has_coarse) MQS_TRY(fold_direct(b->dplain, b->n, 1, 0));
      }
      // a non-positive pivot in any factor of the sample
      std::vector<int32_t> h((size_t)b->n);
      for (auto& f : b->fsets) {
        MQS_CUDA_TRY(cudaMemcpyAsync(h.data(), f->bad.p, h.size() * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st));
        MQS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int s2 = 0; s2 < b->n; ++s2)
          if (h[s2]) out[s2] |= MQS_ST_NOTSPD;
      }
    }
    MQS_CUDA_TRY(cudaMemcpyAsync(status, out.data(), out.size() * sizeof(int32_t),
                                 cudaMemcpyDefault, st));
  }
  MQS_CUDA_TRY(cudaStreamSynchronize(st));
  return MQS_OK;
}

int mqs_read_state(mqs_ctx* ctx, int32_t batch_id, int32_t which, double* a) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (!a || (which != 0 && which != 1) || b->mode == 0 || (which == 1 && !b->has_coarse)) {
    set_error("no such state (which = %d)", which);
    return MQS_EINVAL;
  }
  const MeshDev& m = *ctx->c.meshes[b->mesh_id];
  const cudaStream_t st = ctx->c.stream;
  const bool dev = is_device_ptr(a);
  DevBuf tmp;
  double* out = a;
  if (!dev) {
    MQS_TRY(tmp.ensure((size_t)b->n * m.n_free * sizeof(double)));
    out = tmp.as<double>();
  }
  if (b->mode >= 3) {
    const size_t row = (size_t)m.n_free * sizeof(double);
    const double* src;
    size_t pitch;
    if (which == 0 && b->mode == 4) {
      src = b->E_final + (size_t)(b->M - 1) * m.n_free;
      pitch = row * b->M;
    } else {
      const int lane0 = which == 0 ? 0 : b->nf_direct;
      src = b->dplain.v(lane0, 0);
      pitch = row * 5;
    }
    MQS_CUDA_TRY(cudaMemcpy2DAsync(out, row, src, pitch, row, b->n, cudaMemcpyDeviceToDevice, st));
  } else if (which == 0 && b->mode == 2) {
    MQS_TRY(transpose_to_rows(b->par.vec(V_A0), b->par.xs, m.n_free, b->n, b->M, b->M - 1, out, st));
  } else if (which == 0) {
    MQS_TRY(transpose_to_rows(b->plain.vec(V_A0), b->plain.xs, m.n_free, b->n, 1, 0, out, st));
  } else {
    const int off = b->mode == 2 ? 0 : b->nf_pad;
    MQS_TRY(transpose_to_rows(b->plain.vec(V_A0), b->plain.xs, m.n_free, b->n, 1, off, out, st));
  }
  if (!dev)
    MQS_CUDA_TRY(cudaMemcpyAsync(a, out, (size_t)b->n * m.n_free * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  MQS_CUDA_TRY(cudaStreamSynchronize(st));
  return MQS_OK;
}

int mqs_read_stats(mqs_ctx* ctx, int32_t batch_id, double* stats) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (!stats) {
    set_error("null stats array");
    return MQS_EINVAL;
  }
  double prop = 0.0, chain = 0.0, t;
  if (b->mode >= 3) {
    // the banded solver has no iterations
  } else if (b->mode == 1 || b->has_coarse) {
    MQS_TRY(sum_host(ctx, b->plain.iters, b->plain.xs, t));
    prop += t;
  }
  if (b->mode == 2) {
    MQS_TRY(sum_host(ctx, b->par.iters, b->par.lanes, t));
    prop += t;
    MQS_TRY(sum_host(ctx, b->chain.iters, b->chain.xs, t));
    chain += t;
  }
  b->stats[0] = prop + chain;
  b->stats[4] = prop;
  b->stats[5] = chain;
  memcpy(stats, b->stats, sizeof(b->stats));
  return MQS_OK;
}

int mqs_profile(mqs_ctx* ctx, int32_t enable) {
  MQS_TRY(enter(ctx));
  ctx->c.prof = enable != 0;
  if (enable) {
    ctx->c.ev_used[0] = ctx->c.ev_used[1] = 0;
    if (!ctx->c.prof_t0) MQS_CUDA_TRY(cudaEventCreate(&ctx->c.prof_t0));
    MQS_CUDA_TRY(cudaEventRecord(ctx->c.prof_t0, ctx->c.stream));
  }
  return MQS_OK;
}

int mqs_profile_read(mqs_ctx* ctx, double* out) {
  MQS_TRY(enter(ctx));
  if (!out) {
    set_error("null output array");
    return MQS_EINVAL;
  }
  MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  out[0] = (double)g_launches.load();
  for (int k = 0; k < 2; ++k) {
    double ms = 0.0;
    std::vector<std::pair<double, double>> iv;
    for (size_t j = 0; j < ctx->c.ev_used[k]; ++j) {
      float e = 0.0f, a = 0.0f, z = 0.0f;
      MQS_CUDA_TRY(cudaEventSynchronize(ctx->c.ev[k][j].second));
      MQS_CUDA_TRY(cudaEventElapsedTime(&e, ctx->c.ev[k][j].first, ctx->c.ev[k][j].second));
      ms += e;
      if (ctx->c.prof_t0) {
        MQS_CUDA_TRY(cudaEventElapsedTime(&a, ctx->c.prof_t0, ctx->c.ev[k][j].first));
        MQS_CUDA_TRY(cudaEventElapsedTime(&z, ctx->c.prof_t0, ctx->c.ev[k][j].second));
        iv.emplace_back(a, z);
      }
    }
    // time covered by at least one launch of the kind (launches on several
    // streams overlap)
    std::sort(iv.begin(), iv.end());
    double covered = 0.0, cur_a = 0.0, cur_z = -1.0;
    for (const auto& x : iv) {
      if (x.first > cur_z) {
        if (cur_z > cur_a) covered += cur_z - cur_a;
        cur_a = x.first;
        cur_z = x.second;
      } else {
        cur_z = std::max(cur_z, x.second);
      }
    }
    if (cur_z > cur_a) covered += cur_z - cur_a;
    out[1 + 2 * k] = (double)ctx->c.ev_used[k];
    out[2 + 2 * k] = ms;
    out[5 + k] = covered;
  }
  return MQS_OK;
}

int mqs_profile_trace(mqs_ctx* ctx, int32_t kind, double* out, int32_t max_launches,
                      int32_t* count) {
  MQS_TRY(enter(ctx));
  if (kind < 0 || kind > 1 || !count || (max_launches > 0 && !out)) {
    set_error("bad arguments to mqs_profile_trace");
    return MQS_EINVAL;
  }
  const Ctx& c = ctx->c;
  *count = (int32_t)c.ev_used[kind];
  if (!c.prof_t0) return MQS_OK;
  MQS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  for (size_t j = 0; j < c.ev_used[kind] && (int64_t)j < max_launches; ++j) {
    float a = 0.0f, z = 0.0f;
    MQS_CUDA_TRY(cudaEventSynchronize(c.ev[kind][j].second));
    MQS_CUDA_TRY(cudaEventElapsedTime(&a, c.prof_t0, c.ev[kind][j].first));
    MQS_CUDA_TRY(cudaEventElapsedTime(&z, c.prof_t0, c.ev[kind][j].second));
    out[2 * j] = a;
    out[2 * j + 1] = z;
  }
  return MQS_OK;
}

int mqs_apply(mqs_ctx* ctx, int32_t batch_id, int32_t which, double dt, const double* x,
              double* y) {
  MQS_TRY(enter(ctx));
  Batch* bp = get_batch(ctx, batch_id);
  if (!bp) return MQS_EINVAL;
  Batch& b = *bp;
  if (!x || !y || which < 0 || which > 2) {
    set_error("bad arguments to mqs_apply");
    return MQS_EINVAL;
  }
  const MeshDev& m = *ctx->c.meshes[b.mesh_id];
  const cudaStream_t st = ctx->c.stream;
  const int saved_kind = b.qoi_kind;
  if (which == 1) b.qoi_kind = MQS_QOI_ENERGY;   // build K values
  int rc = ensure_mk(ctx, b, m);
  b.qoi_kind = saved_kind;
  if (rc != MQS_OK) return rc;
  const double* vals = nullptr;
  if (which == 0) vals = b.Mv.as<double>();
  if (which == 1) vals = b.Kv.as<double>();
  if (which == 2) {
    ValueSet* v = value_set(ctx, b, m, dt, false, rc);
    if (!v) return rc;
    vals = v->A.as<double>();
  }
  const size_t bytes = (size_t)b.n * m.n_free * sizeof(double);
  DevBuf dx, dy;
  const double* xin = x;
  double* yout = y;
  if (!is_device_ptr(x)) {
    MQS_TRY(dx.ensure(bytes));
    MQS_CUDA_TRY(cudaMemcpyAsync(dx.p, x, bytes, cudaMemcpyHostToDevice, st));
    xin = dx.as<double>();
  }
  const bool ydev = is_device_ptr(y);
  if (!ydev) {
    MQS_TRY(dy.ensure(bytes));
    yout = dy.as<double>();
  }
  MQS_TRY(batched_spmv(m, vals, b.n, b.n, xin, yout, st));
  if (!ydev) MQS_CUDA_TRY(cudaMemcpyAsync(y, yout, bytes, cudaMemcpyDeviceToHost, st));
  MQS_CUDA_TRY(cudaStreamSynchronize(st));
  return MQS_OK;
}

int mqs_mlmc_reset(mqs_ctx* ctx, int32_t n_levels) {
  MQS_TRY(enter(ctx));
  if (n_levels < 1 || n_levels > 64) {
    set_error("n_levels = %d out of range [1, 64]", n_levels);
    return MQS_EINVAL;
  }
  MQS_TRY(ctx->c.mlmc.ensure((size_t)n_levels * 4 * sizeof(double)));
  MQS_CUDA_TRY(cudaMemsetAsync(ctx->c.mlmc.p, 0, (size_t)n_levels * 4 * sizeof(double),
                               ctx->c.stream));
  ctx->c.n_levels = n_levels;
  return MQS_OK;
}

int mqs_mlmc_accumulate(mqs_ctx* ctx, int32_t batch_id, int32_t level) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  if (level < 0 || level >= ctx->c.n_levels || b->mode == 0) {
    set_error("level %d outside the %d reset levels, or batch not propagated", level,
              ctx->c.n_levels);
    return MQS_EINVAL;
  }
  return mlmc_accumulate_dev(b->qoi.as<double>(), b->n, level,
                             ctx->c.mlmc.as<double>() + 4 * level, ctx->c.stream);
}

int mqs_mlmc_readout(mqs_ctx* ctx, double* levels, double* estimate, double* rmse) {
  MQS_TRY(enter(ctx));
  if (ctx->c.n_levels < 1) {
    set_error("mqs_mlmc_reset was not called");
    return MQS_EINVAL;
  }
  std::vector<double> rec((size_t)ctx->c.n_levels * 4);
  MQS_CUDA_TRY(cudaMemcpyAsync(rec.data(), ctx->c.mlmc.p, rec.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->c.stream));
  MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  double est = 0.0, var_sum = 0.0;
  for (int l = 0; l < ctx->c.n_levels; ++l) {
    const double n = rec[4 * l], mean = rec[4 * l + 1], m2 = rec[4 * l + 2];
    const double var = n > 1.0 ? m2 / (n - 1.0) : 0.0;
    if (levels) {
      levels[3 * l] = n;
      levels[3 * l + 1] = mean;
      levels[3 * l + 2] = var;
    }
    est += mean;
    if (n > 0.0) var_sum += var / n;
  }
  if (estimate) *estimate = est;
  if (rmse) *rmse = std::sqrt(var_sum);
  return MQS_OK;
}

int mqs_lane_slots(mqs_ctx* ctx, int32_t precision, int32_t* slots) {
  MQS_TRY(enter(ctx));
  if (!slots || (precision != MQS_FP64 && precision != MQS_MIXED)) {
    set_error("bad arguments to mqs_lane_slots");
    return MQS_EINVAL;
  }
  const int r = direct_lane_slots(precision == MQS_MIXED ? 1 : 0);
  if (r < 0) return MQS_ECUDA;
  *slots = r;
  return MQS_OK;
}

int mqs_set_test_hook(mqs_ctx* ctx, int32_t hook) {
  MQS_TRY(enter(ctx));
  if (hook != 0 && hook != MQS_TEST_HOOK_STALL) {
    set_error("unknown test hook %d", hook);
    return MQS_EINVAL;
  }
  ctx->c.test_hook = hook;
  return MQS_OK;
}

int mqs_free_batch(mqs_ctx* ctx, int32_t batch_id) {
  MQS_TRY(enter(ctx));
  Batch* b = get_batch(ctx, batch_id);
  if (!b) return MQS_EINVAL;
  MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  ctx->c.meshes[b->mesh_id]->live_batches--;
  ctx->c.batches[batch_id].reset();
  return MQS_OK;
}

int mqs_free_mesh(mqs_ctx* ctx, int32_t mesh_id) {
  MQS_TRY(enter(ctx));
  MeshDev* m = get_mesh(ctx, mesh_id);
  if (!m) return MQS_EINVAL;
  if (m->live_batches > 0) {
    set_error("mesh %d still has %d live batches", mesh_id, m->live_batches);
    return MQS_EINVAL;
  }
  MQS_CUDA_TRY(cudaStreamSynchronize(ctx->c.stream));
  ctx->c.meshes[mesh_id].reset();
  return MQS_OK;
}

}  // extern "C"
