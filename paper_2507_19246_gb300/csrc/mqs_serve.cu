// Request server: continuous batching of sample solves on one GPU.
//
// Requests are MLMC level samples (the level-l solve from a(t0) = 0 and, if
// asked, the level-(l-1) companion on the same parameters, Eq. 9) or Parareal
// slices (one fine propagation from a given state over steps [k0, k0 + n),
// the F of Eq. 12), on any uploaded mesh and with any step count.  They wait
// in arrival order.  Each call of mqs_server_progress
//  * detects finished requests: every lane writes its QoI and status to
//    host-mapped memory and then raises a done flag (system-scope release),
//    so a request completes as soon as its own lanes have, not when its batch
//    does;
//  * releases the device memory of batches whose stream has drained;
//  * if a stream is free, admits queued requests in arrival order while their
//    device footprint (values, factors, lane vectors) fits the HBM budget and
//    launches them as one batch on that stream: per-sample values, band
//    Cholesky factors for every lane's step size, then the stepping kernel
//    over all lanes of a mesh.
// Batches on different streams run at the same time, so requests admitted
// while others are on the GPU start without waiting for them: their CTAs
// take SMs as the running lanes release them.  Every lane runs the same
// launch shape (one 256-thread CTA, work vector in L2) whatever the batch, so
// a request's result does not depend on what it is batched with.  Device
// memory of a batch is one stream-ordered allocation, freed on its stream.
#include "mqs_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>

namespace mqs {
namespace {

constexpr double kTwoPi = 6.28318530717958647692;

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

struct Request {
  int64_t id = 0;
  int mesh_id = 0, kind = 0, qoi_kind = 0, lanes = 1;
  std::vector<double> params, a_init;
  double* a_out = nullptr;            // device, caller-owned (slice final state), or null
  double t0 = 0.0, dt = 0.0, dt_prev = 0.0;
  int n_steps = 0, n_steps_prev = 0;
  int64_t k0 = 0;
  size_t bytes = 0;
  int slot = -1;                      // result slot in mapped memory
  bool finished = false;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

struct Run {
  int stream = -1;
  cudaEvent_t ev = nullptr;
  size_t bytes = 0;
  std::vector<int64_t> ids;
};

// Per-lane device footprint pieces of a request on mesh m.
struct Footprint {
  size_t per_request, per_lane;
};

Footprint footprint(const MeshDev& m, int qoi_kind) {
  const size_t n = (size_t)m.n_free, z = (size_t)m.nnz;
  const size_t nblk = (n + 31) / 32;
  Footprint f;
  f.per_request = al((size_t)(2 * m.n_regions + 1 + 2 * m.n_phases) * sizeof(double)) +
                  al(z * sizeof(double)) + (qoi_kind == MQS_QOI_ENERGY ? al(z * sizeof(double)) : 0);
  f.per_lane = al(z * sizeof(double)) +                              // A values (factor input)
               al(n * (m.bw + 1) * sizeof(double)) + al(n * sizeof(double)) +   // factor, 1/diag
               al(nblk * 32 * 32 * sizeof(double)) + al(sizeof(int32_t)) +      // block inverses, flag
               5 * al(n * sizeof(double)) +                           // a0, a1, y, w, b
               al(sizeof(DirectLane));
  return f;
}

}  // namespace
}  // namespace mqs

using namespace mqs;

struct mqs_server {
  mqs_ctx* ctx = nullptr;
  int device = 0;
  int64_t budget = 0, used = 0;
  int max_lanes = 0;
  double freq = 50.0;
  std::vector<cudaStream_t> streams;
  std::vector<bool> busy;
  std::deque<Request*> queue;
  std::map<int64_t, std::unique_ptr<Request>> live;
  std::vector<Run> runs;
  // result slots in host-mapped memory: qoi[2], status[2], done[2] per slot
  int n_slots = 0;
  double* qoi_h = nullptr;
  int32_t* st_h = nullptr;
  int32_t* done_h = nullptr;
  double* qoi_d = nullptr;
  int32_t* st_d = nullptr;
  int32_t* done_d = nullptr;
  std::vector<int> free_slots;
  struct Done {
    int64_t id;
    double qoi[2];
    int32_t status;
    double t[3];
  };
  std::deque<Done> completed;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t_origin = std::chrono::steady_clock::now();

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_origin).count();
  }
  ~mqs_server() {
    cudaSetDevice(device);
    for (cudaStream_t s : streams) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    for (Run& r : runs)
      if (r.ev) cudaEventDestroy(r.ev);
    if (qoi_h) cudaFreeHost(qoi_h);
    if (st_h) cudaFreeHost(st_h);
    if (done_h) cudaFreeHost(done_h);
  }
};

namespace {

int launch_batch(mqs_server& S, int stream_idx, std::vector<Request*>& batch) {
  const cudaStream_t st = S.streams[stream_idx];
  // lay out one allocation: per (mesh, qoi kind) group the request and lane pieces
  struct Group {
    const MeshDev* m;
    int qoi_kind;
    std::vector<Request*> reqs;
  };
  std::vector<Group> groups;
  for (Request* r : batch) {
    const MeshDev* m = ctx_mesh(S.ctx, r->mesh_id);
    auto it = std::find_if(groups.begin(), groups.end(), [&](const Group& g) {
      return g.m == m && g.qoi_kind == r->qoi_kind;
    });
    if (it == groups.end()) {
      groups.push_back(Group{m, r->qoi_kind, {}});
      it = groups.end() - 1;
    }
    it->reqs.push_back(r);
  }
  size_t total = 0;
  for (Request* r : batch) total += r->bytes;
  unsigned char* block = nullptr;
  MQS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&block), std::max<size_t>(total, 256), st));
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* p = block + off;
    off += al(b);
    return p;
  };
  for (Group& g : groups) {
    const MeshDev& m = *g.m;
    const int R = (int)g.reqs.size();
    const int np = 2 * m.n_regions + 1 + 2 * m.n_phases;
    int G = 0;
    for (Request* r : g.reqs) G += r->lanes;
    const size_t n = (size_t)m.n_free, z = (size_t)m.nnz, nblk = (n + 31) / 32;
    auto* params = reinterpret_cast<double*>(take((size_t)R * np * sizeof(double)));
    auto* Mv = reinterpret_cast<double*>(take((size_t)R * z * sizeof(double)));
    double* Kv = g.qoi_kind == MQS_QOI_ENERGY
                     ? reinterpret_cast<double*>(take((size_t)R * z * sizeof(double)))
                     : nullptr;
    auto* Av = reinterpret_cast<double*>(take((size_t)G * z * sizeof(double)));
    const size_t fstride = n * (m.bw + 1);
    auto* LB = reinterpret_cast<double*>(take((size_t)G * fstride * sizeof(double)));
    auto* invd = reinterpret_cast<double*>(take((size_t)G * n * sizeof(double)));
    auto* Binv = reinterpret_cast<double*>(take((size_t)G * nblk * 1024 * sizeof(double)));
    auto* bad = reinterpret_cast<int32_t*>(take((size_t)G * sizeof(int32_t)));
    auto* vec = reinterpret_cast<double*>(take((size_t)G * 5 * n * sizeof(double)));
    auto* desc = reinterpret_cast<DirectLane*>(take((size_t)G * sizeof(DirectLane)));
    if (off > total) {   // the group layout never needs more than the footprints
      set_error("internal: server batch layout exceeds its allocation");
      cudaFreeAsync(block, st);
      return MQS_ECUDA;
    }
    std::vector<double> hp((size_t)R * np);
    for (int r = 0; r < R; ++r) std::copy(g.reqs[r]->params.begin(), g.reqs[r]->params.end(),
                                          hp.begin() + (size_t)r * np);
    MQS_CUDA_TRY(cudaMemcpyAsync(params, hp.data(), hp.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
    // M (and K) of every sample; A = M/dt + K of every lane's step size
    MQS_TRY(expand_values(m, params, R, np, 1.0, R, nullptr, Mv, Kv, nullptr, nullptr, nullptr, R,
                          st));
    std::vector<DirectLane> hd((size_t)G);
    int j = 0;
    for (int r = 0; r < R; ++r) {
      Request& q = *g.reqs[r];
      for (int lane = 0; lane < q.lanes; ++lane, ++j) {
        const double dt = lane == 0 ? q.dt : q.dt_prev;
        const int steps = lane == 0 ? q.n_steps : q.n_steps_prev;
        MQS_TRY(expand_values(m, params + (size_t)r * np, 1, np, dt, G, Av + j, nullptr, nullptr,
                              nullptr, nullptr, nullptr, G, st));
        DirectLane& d = hd[(size_t)j];
        memset(&d, 0, sizeof(d));
        d.LB = LB + (size_t)j * fstride;
        d.invd = invd + (size_t)j * n;
        d.Binv = Binv + (size_t)j * nblk * 1024;
        double* v = vec + (size_t)j * 5 * n;
        const bool caller_state = q.kind == MQS_REQ_SLICE && q.a_out;
        d.a0 = caller_state ? q.a_out : v;
        d.a1 = v + n;
        d.y = v + 2 * n;
        d.w = v + 3 * n;
        d.b = v + 4 * n;
        d.status_out = S.st_d + 2 * q.slot + lane;
        d.qoi_out = S.qoi_d + 2 * q.slot + lane;
        d.done_flag = S.done_d + 2 * q.slot + lane;
        // a level solve returns the finished QoI (Eq. 26: / T; energy: / N),
        // a slice its raw partial sum (what Parareal adds over the slices)
        d.qoi_scale = q.kind == MQS_REQ_SLICE ? 1.0
                      : (q.qoi_kind == MQS_QOI_JOULE ? 1.0 / ((double)steps * dt) : 1.0 / steps);
        d.vcol = r;
        const double* p = q.params.data();
        for (int ph = 0; ph < kMaxPhases; ++ph) {
          d.amp[ph] = ph < m.n_phases ? p[2 * m.n_regions] * p[2 * m.n_regions + 1 + ph] : 0.0;
          d.phase[ph] = ph < m.n_phases ? p[2 * m.n_regions + 1 + m.n_phases + ph] : 0.0;
        }
        d.dt = dt;
        d.t0 = q.t0;
        d.k0 = q.kind == MQS_REQ_SLICE ? q.k0 : 0;
        d.n_steps = steps;
        d.init_from_a0 = (q.kind == MQS_REQ_SLICE && !q.a_init.empty()) ? 1 : 0;
        d.sample = r;
        if (d.init_from_a0)
          MQS_CUDA_TRY(cudaMemcpyAsync(d.a0, q.a_init.data(), n * sizeof(double),
                                       cudaMemcpyHostToDevice, st));
      }
    }
    MQS_TRY(band_factor<double>(m, Av, G, G, LB, invd, Binv, bad, st));
    MQS_CUDA_TRY(cudaMemcpyAsync(desc, hd.data(), hd.size() * sizeof(DirectLane),
                                 cudaMemcpyHostToDevice, st));
    DirectConst kc;
    memset(&kc, 0, sizeof(kc));
    kc.rowptr = m.rowptr.as<int32_t>();
    kc.colidx = m.colidx.as<int32_t>();
    kc.iperm = m.iperm.as<int32_t>();
    kc.perm = m.perm.as<int32_t>();
    kc.M = Mv;
    kc.K = Kv;
    kc.vs = R;
    kc.F = m.F.as<double>();
    kc.n = m.n_free;
    kc.bw = m.bw;
    kc.n_phases = m.n_phases;
    kc.qoi_kind = g.qoi_kind;
    kc.omega = kTwoPi * S.freq;
    kc.w_in_smem = 0;   // one launch shape for every batch: 256 threads, work vector in L2
    kc.max_sweeps = 1;
    MQS_TRY(launch_direct(desc, G, kc, st));
  }
  Run run;
  run.stream = stream_idx;
  run.bytes = total;
  for (Request* r : batch) run.ids.push_back(r->id);
  MQS_CUDA_TRY(cudaEventCreateWithFlags(&run.ev, cudaEventDisableTiming));
  MQS_CUDA_TRY(cudaEventRecord(run.ev, st));
  MQS_CUDA_TRY(cudaFreeAsync(block, st));
  S.runs.push_back(run);
  S.busy[stream_idx] = true;
  S.used += (int64_t)total;
  return MQS_OK;
}

}  // namespace

extern "C" {

int mqs_server_create(mqs_ctx* ctx, int64_t hbm_budget, int32_t n_streams, int32_t max_batch_lanes,
                      double freq_hz, mqs_server** out) {
  clear_error();
  if (!ctx || !out || n_streams < 1 || n_streams > 32 || max_batch_lanes < 1 ||
      !(freq_hz > 0.0) || !std::isfinite(freq_hz)) {
    set_error("bad arguments to mqs_server_create");
    return MQS_EINVAL;
  }
  auto srv = std::unique_ptr<mqs_server>(new mqs_server());
  srv->ctx = ctx;
  srv->device = ctx_device(ctx);
  MQS_CUDA_TRY(cudaSetDevice(srv->device));
  if (hbm_budget <= 0) {
    size_t fr = 0, tot = 0;
    MQS_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    hbm_budget = (int64_t)(0.8 * (double)fr);
  }
  srv->budget = hbm_budget;
  srv->max_lanes = max_batch_lanes;
  srv->freq = freq_hz;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t s;
    MQS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    srv->streams.push_back(s);
    srv->busy.push_back(false);
  }
  srv->n_slots = 4 * max_batch_lanes * n_streams;
  MQS_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&srv->qoi_h),
                             (size_t)srv->n_slots * 2 * sizeof(double), cudaHostAllocMapped));
  MQS_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&srv->st_h),
                             (size_t)srv->n_slots * 2 * sizeof(int32_t), cudaHostAllocMapped));
  MQS_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&srv->done_h),
                             (size_t)srv->n_slots * 2 * sizeof(int32_t), cudaHostAllocMapped));
  MQS_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&srv->qoi_d), srv->qoi_h, 0));
  MQS_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&srv->st_d), srv->st_h, 0));
  MQS_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&srv->done_d), srv->done_h, 0));
  for (int i = srv->n_slots - 1; i >= 0; --i) srv->free_slots.push_back(i);
  *out = srv.release();
  return MQS_OK;
}

int mqs_server_destroy(mqs_server* srv) {
  delete srv;
  return MQS_OK;
}

int mqs_server_submit(mqs_server* srv, int32_t mesh_id, int32_t n_params, const double* params,
                      int32_t kind, int32_t qoi_kind, double t0, double dt, int32_t n_steps,
                      double dt_prev, int32_t n_steps_prev, int64_t k0, const double* a_init,
                      double* a_out, int64_t* request_id) {
  clear_error();
  if (!srv || !params || !request_id) {
    set_error("null argument");
    return MQS_EINVAL;
  }
  const MeshDev* m = ctx_mesh(srv->ctx, mesh_id);
  if (!m) {
    set_error("invalid mesh id %d", mesh_id);
    return MQS_EINVAL;
  }
  if (m->bw < 0) {
    set_error("mesh %d has no band ordering", mesh_id);
    return MQS_EINVAL;
  }
  const int np = 2 * m->n_regions + 1 + 2 * m->n_phases;
  if (n_params != np || (kind != MQS_REQ_LEVEL && kind != MQS_REQ_SLICE) ||
      (qoi_kind != MQS_QOI_JOULE && qoi_kind != MQS_QOI_ENERGY) || !(dt > 0.0) || n_steps < 1 ||
      (kind == MQS_REQ_LEVEL && dt_prev > 0.0 && n_steps_prev < 1) || k0 < 0 ||
      (kind == MQS_REQ_LEVEL && (a_init || a_out))) {
    set_error("bad request: n_params %d (mesh needs %d), kind %d, qoi %d, dt %g, steps %d, "
              "dt_prev %g, steps_prev %d, k0 %lld",
              n_params, np, kind, qoi_kind, dt, n_steps, dt_prev, n_steps_prev, (long long)k0);
    return MQS_EINVAL;
  }
  auto r = std::unique_ptr<Request>(new Request());
  r->id = srv->next_id++;
  r->mesh_id = mesh_id;
  r->kind = kind;
  r->qoi_kind = qoi_kind;
  r->lanes = (kind == MQS_REQ_LEVEL && dt_prev > 0.0) ? 2 : 1;
  r->params.assign(params, params + np);
  if (a_init) r->a_init.assign(a_init, a_init + m->n_free);
  r->a_out = a_out;
  r->t0 = t0;
  r->dt = dt;
  r->n_steps = n_steps;
  r->dt_prev = r->lanes == 2 ? dt_prev : 0.0;
  r->n_steps_prev = r->lanes == 2 ? n_steps_prev : 0;
  r->k0 = k0;
  const Footprint f = footprint(*m, qoi_kind);
  r->bytes = f.per_request + r->lanes * f.per_lane;
  if ((int64_t)r->bytes > srv->budget) {
    set_error("request needs %zu bytes of device memory, more than the server's budget of %lld",
              r->bytes, (long long)srv->budget);
    return MQS_EINVAL;
  }
  r->t_submit = srv->now();
  *request_id = r->id;
  srv->queue.push_back(r.get());
  srv->live[r->id] = std::move(r);
  return MQS_OK;
}

int mqs_server_footprint(mqs_server* srv, int32_t mesh_id, int32_t qoi_kind, int32_t lanes,
                         int64_t* bytes) {
  clear_error();
  const MeshDev* m = srv ? ctx_mesh(srv->ctx, mesh_id) : nullptr;
  if (!m || !bytes || lanes < 1 || lanes > 2) {
    set_error("bad arguments to mqs_server_footprint");
    return MQS_EINVAL;
  }
  const Footprint f = footprint(*m, qoi_kind);
  *bytes = (int64_t)(f.per_request + lanes * f.per_lane);
  return MQS_OK;
}

int mqs_server_progress(mqs_server* srv, int32_t* in_flight, int32_t* queued) {
  clear_error();
  if (!srv) {
    set_error("null server");
    return MQS_EINVAL;
  }
  MQS_CUDA_TRY(cudaSetDevice(srv->device));
  // a request is complete once all its lanes have raised their done flag
  auto complete = [&](Request& r) {
    if (r.slot < 0 || r.finished) return;
    for (int l = 0; l < r.lanes; ++l)
      if (reinterpret_cast<volatile int32_t*>(srv->done_h)[2 * r.slot + l] == 0) return;
    std::atomic_thread_fence(std::memory_order_acquire);
    r.finished = true;
    r.t_done = srv->now();
    mqs_server::Done d;
    d.id = r.id;
    d.qoi[0] = srv->qoi_h[2 * r.slot];
    d.qoi[1] = r.lanes == 2 ? srv->qoi_h[2 * r.slot + 1] : 0.0;
    d.status = srv->st_h[2 * r.slot] | (r.lanes == 2 ? srv->st_h[2 * r.slot + 1] : 0);
    d.t[0] = r.t_submit;
    d.t[1] = r.t_admit;
    d.t[2] = r.t_done;
    srv->completed.push_back(d);
  };
  // (1) finished requests
  for (auto& kv : srv->live) complete(*kv.second);
  // (2) batches whose stream has drained (every lane ended, so every flag is
  // set): device memory, the stream and the result slots are released
  std::vector<Run> keep;
  for (Run& run : srv->runs) {
    const cudaError_t e = cudaEventQuery(run.ev);
    if (e == cudaErrorNotReady) {
      keep.push_back(run);
      continue;
    }
    if (e != cudaSuccess) {
      set_error("a server batch failed: %s", cudaGetErrorString(e));
      return MQS_ECUDA;
    }
    cudaEventDestroy(run.ev);
    srv->used -= (int64_t)run.bytes;
    srv->busy[run.stream] = false;
    for (int64_t id : run.ids) {
      auto it = srv->live.find(id);
      if (it == srv->live.end()) continue;
      complete(*it->second);
      srv->free_slots.push_back(it->second->slot);
      srv->live.erase(it);
    }
  }
  srv->runs.swap(keep);
  // (3) admit queued requests in arrival order into one batch per free stream
  for (size_t si = 0; si < srv->streams.size() && !srv->queue.empty(); ++si) {
    if (srv->busy[si]) continue;
    std::vector<Request*> batch;
    int64_t bytes = 0;
    int lanes = 0;
    while (!srv->queue.empty()) {
      Request* r = srv->queue.front();
      if (srv->used + bytes + (int64_t)r->bytes > srv->budget) break;
      if (lanes + r->lanes > srv->max_lanes && !batch.empty()) break;
      if (srv->free_slots.empty()) break;
      r->slot = srv->free_slots.back();
      srv->free_slots.pop_back();
      for (int l = 0; l < 2; ++l) {
        srv->done_h[2 * r->slot + l] = 0;
        srv->st_h[2 * r->slot + l] = 0;
        srv->qoi_h[2 * r->slot + l] = 0.0;
      }
      r->t_admit = srv->now();
      bytes += (int64_t)r->bytes;
      lanes += r->lanes;
      batch.push_back(r);
      srv->queue.pop_front();
    }
    if (batch.empty()) break;
    std::atomic_thread_fence(std::memory_order_release);
    MQS_TRY(launch_batch(*srv, (int)si, batch));
  }
  if (in_flight) *in_flight = (int32_t)(srv->live.size() - srv->queue.size());
  if (queued) *queued = (int32_t)srv->queue.size();
  return MQS_OK;
}

int mqs_server_poll(mqs_server* srv, int32_t max, int64_t* ids, double* qoi, int32_t* status,
                    double* times, int32_t* count) {
  clear_error();
  if (!srv || !count || (max > 0 && (!ids || !qoi))) {
    set_error("bad arguments to mqs_server_poll");
    return MQS_EINVAL;
  }
  int c = 0;
  while (c < max && !srv->completed.empty()) {
    const mqs_server::Done& d = srv->completed.front();
    ids[c] = d.id;
    qoi[2 * c] = d.qoi[0];
    qoi[2 * c + 1] = d.qoi[1];
    if (status) status[c] = d.status;
    if (times)
      for (int k = 0; k < 3; ++k) times[3 * c + k] = d.t[k];
    srv->completed.pop_front();
    ++c;
  }
  *count = c;
  return MQS_OK;
}

}  // extern "C"
