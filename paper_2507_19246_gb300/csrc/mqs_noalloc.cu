// Allocation-free entry point: sequential implicit-Euler stepping of a batch
// of lanes whose matrices the caller already holds in device memory, with all
// intermediate vectors in a fixed-size static device array instead of memory
// from cudaMalloc.
//
// Who needs it: code that must not allocate device memory while it runs --
// for example a host application that hands the GPU to this library from a
// real-time or signal-safe context (cudaMalloc may block or take locks), or a
// runtime whose device memory is fully carved up by its own pool at start-up
// (a cudaMalloc would fail or fight that pool).  Such callers pass their own
// inputs and outputs and let the library work in this preallocated scratch.
#include "mqs_internal.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace mqs {
namespace {

// 32 MiB of scratch, resident on every GPU that loads the library until the
// process exits.  Holds the tile descriptors, the per-lane bookkeeping and six
// lane vectors of n x n_lanes doubles.
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;
constexpr int kMaxTiles = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
int scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                cudaGetErrorString(e));
      return MQS_ECUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return MQS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// [n_lanes][P] host-order amplitude/phase (already copied to scratch) into the
// [n_lanes][kMaxPhases] lane layout of the stepping kernel, zero padded.
__global__ void k_lane_layout(const double* __restrict__ amp_in, const double* __restrict__ ph_in,
                              int n_lanes, int P, double* __restrict__ amp,
                              double* __restrict__ phi) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_lanes) return;
  for (int q = 0; q < kMaxPhases; ++q) {
    amp[(int64_t)l * kMaxPhases + q] = q < P ? amp_in[(int64_t)l * P + q] : 0.0;
    phi[(int64_t)l * kMaxPhases + q] = q < P ? ph_in[(int64_t)l * P + q] : 0.0;
  }
}

__global__ void k_scale_qoi(const double* __restrict__ raw, int n_lanes, double scale,
                            double* __restrict__ qoi) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_lanes) qoi[l] = raw[l] * scale;
}

}  // namespace
}  // namespace mqs

using namespace mqs;

namespace {

// Restores the calling thread's current device when the entry point returns.
struct DeviceGuard {
  int saved = -1;
  ~DeviceGuard() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

}  // namespace

extern "C" int mqs_propagate_noalloc(int32_t device, void* cuda_stream, int32_t n,
                                     const int32_t* rowptr, const int32_t* colidx, int64_t nnz,
                                     int32_t n_lanes, const double* A, const double* M,
                                     const double* K, const double* Dinv, int32_t n_phases,
                                     const double* F, const double* src_amp,
                                     const double* src_phase, double t0, double dt,
                                     int32_t n_steps, double freq_hz, int32_t qoi_kind,
                                     double cg_tol, int32_t cg_max_iters, double* a_out,
                                     double* qoi_out, int32_t* status_out) {
  clear_error();
  int count = 0;
  MQS_CUDA_TRY(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count || device >= kMaxDevices) {
    set_error("device %d out of range", device);
    return MQS_EINVAL;
  }
  if (n < 1 || nnz < 1 || n_lanes < 1 || n_steps < 1 || !(dt > 0.0) || cg_max_iters < 1 ||
      !(cg_tol >= 0.0) || n_phases < 0 || n_phases > kMaxPhases ||
      (qoi_kind != MQS_QOI_JOULE && qoi_kind != MQS_QOI_ENERGY)) {
    set_error("bad sizes: n %d, nnz %lld, lanes %d, steps %d, dt %g, cg_max_iters %d, phases %d, "
              "qoi %d", n, (long long)nnz, n_lanes, n_steps, dt, cg_max_iters, n_phases, qoi_kind);
    return MQS_EINVAL;
  }
  if (!rowptr || !colidx || !A || !M || !Dinv || !a_out || !qoi_out ||
      (n_phases > 0 && (!F || !src_amp || !src_phase)) ||
      (qoi_kind == MQS_QOI_ENERGY && !K)) {
    set_error("null array argument");
    return MQS_EINVAL;
  }
  // scratch layout
  const size_t lanes = (size_t)n_lanes;
  const size_t vec_bytes = align256((size_t)n * lanes * sizeof(double));
  size_t off = 0;
  const size_t off_tiles = off;
  off += align256(kMaxTiles * sizeof(TileDesc));
  const size_t off_amp_in = off;
  off += align256(lanes * kMaxPhases * sizeof(double));
  const size_t off_ph_in = off;
  off += align256(lanes * kMaxPhases * sizeof(double));
  const size_t off_amp = off;
  off += align256(lanes * kMaxPhases * sizeof(double));
  const size_t off_phi = off;
  off += align256(lanes * kMaxPhases * sizeof(double));
  const size_t off_k0 = off;
  off += align256(lanes * sizeof(int32_t));
  const size_t off_qraw = off;
  off += align256(lanes * sizeof(double));
  const size_t off_status = off;
  off += align256(lanes * sizeof(int32_t));
  const size_t off_iters = off;
  off += align256(lanes * sizeof(double));
  const size_t off_vec = off;
  off += 6 * vec_bytes;
  if (off > kScratchBytes) {
    set_error("problem too large for the no-allocation scratch: needs %zu bytes "
              "(6 x n x n_lanes doubles + bookkeeping), the limit is %zu bytes",
              off, kScratchBytes);
    return MQS_EINVAL;
  }
  DeviceGuard guard;
  MQS_CUDA_TRY(cudaGetDevice(&guard.saved));
  MQS_CUDA_TRY(cudaSetDevice(device));
  unsigned char* base = nullptr;
  MQS_TRY(scratch_address(device, &base));
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // lane tile and cluster shape
  int lanes_p2 = 1;
  while (lanes_p2 < n_lanes && lanes_p2 < 32) lanes_p2 <<= 1;
  const int L = lanes_p2;
  const int n_tiles = (n_lanes + L - 1) / L;
  if (n_tiles > kMaxTiles) {
    set_error("too many lane tiles (%d, limit %d)", n_tiles, kMaxTiles);
    return MQS_EINVAL;
  }
  const int c_rows = std::max(1, n / (team_threads() / L));
  const int C = std::max(1, std::min(max_cluster(L, MQS_FP64, 0), c_rows));

  // per-call state that must start at zero or from the inputs
  auto* amp_in = reinterpret_cast<double*>(base + off_amp_in);
  auto* ph_in = reinterpret_cast<double*>(base + off_ph_in);
  auto* amp = reinterpret_cast<double*>(base + off_amp);
  auto* phi = reinterpret_cast<double*>(base + off_phi);
  auto* k0 = reinterpret_cast<int32_t*>(base + off_k0);
  auto* qraw = reinterpret_cast<double*>(base + off_qraw);
  auto* iters = reinterpret_cast<double*>(base + off_iters);
  int32_t* status = status_out ? status_out : reinterpret_cast<int32_t*>(base + off_status);
  MQS_CUDA_TRY(cudaMemsetAsync(k0, 0, lanes * sizeof(int32_t), st));
  MQS_CUDA_TRY(cudaMemsetAsync(qraw, 0, lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(iters, 0, lanes * sizeof(double), st));
  MQS_CUDA_TRY(cudaMemsetAsync(status, 0, lanes * sizeof(int32_t), st));
  if (n_phases > 0) {
    MQS_CUDA_TRY(cudaMemcpyAsync(amp_in, src_amp, lanes * n_phases * sizeof(double),
                                 cudaMemcpyDefault, st));
    MQS_CUDA_TRY(cudaMemcpyAsync(ph_in, src_phase, lanes * n_phases * sizeof(double),
                                 cudaMemcpyDefault, st));
  }
  k_lane_layout<<<(n_lanes + 127) / 128, 128, 0, st>>>(amp_in, ph_in, n_lanes, n_phases, amp, phi);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();

  // tile descriptors: lane vectors share the stride n_lanes with a_out
  TileDesc tiles[kMaxTiles];
  double* vec = reinterpret_cast<double*>(base + off_vec);
  auto vptr = [&](int j) { return reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(vec) + j * vec_bytes); };
  for (int t = 0; t < n_tiles; ++t) {
    TileDesc& d = tiles[t];
    memset(&d, 0, sizeof(d));
    const int l0 = t * L;
    d.A = A + l0;
    d.M = M + l0;
    d.K = K ? K + l0 : nullptr;
    d.Dinv = Dinv + l0;
    d.vs = n_lanes;
    d.ds = n_lanes;
    d.ls = 1;
    d.lane0 = l0;
    d.a0 = a_out + l0;
    d.a1 = vptr(0) + l0;
    d.y = vptr(1) + l0;
    d.r = vptr(2) + l0;
    d.p = vptr(3) + l0;
    d.q = vptr(4) + l0;
    d.z = vptr(5) + l0;
    d.xs = n_lanes;
    d.dt = dt;
    d.t0 = t0;
    d.n_steps = n_steps;
    d.n_active = std::min(L, n_lanes - l0);
    d.init_from_a0 = 0;
  }
  auto* d_tiles = reinterpret_cast<TileDesc*>(base + off_tiles);
  MQS_CUDA_TRY(cudaMemcpyAsync(d_tiles, tiles, n_tiles * sizeof(TileDesc), cudaMemcpyHostToDevice,
                               st));
  TeamConst kc;
  memset(&kc, 0, sizeof(kc));
  kc.rowptr = rowptr;
  kc.colidx = colidx;
  kc.F = F;
  kc.n = n;
  kc.n_phases = n_phases;
  kc.qoi_kind = qoi_kind;
  kc.max_it = cg_max_iters;
  kc.replace_every = 50;
  kc.tol2 = cg_tol * cg_tol;
  kc.omega = 6.28318530717958647692 * freq_hz;
  kc.lanes = LaneArrays{amp, phi, k0, qraw, status, iters};
  MQS_TRY(launch_propagate(d_tiles, n_tiles, L, C, MQS_FP64, kc, st));
  const double scale = qoi_kind == MQS_QOI_JOULE ? 1.0 / ((double)n_steps * dt) : 1.0 / n_steps;
  k_scale_qoi<<<(n_lanes + 127) / 128, 128, 0, st>>>(qraw, n_lanes, scale, qoi_out);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}
