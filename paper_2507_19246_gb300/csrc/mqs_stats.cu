// Small kernels around the team kernels: lane bookkeeping for Parareal,
// layout changes at the API boundary, QoI normalisation and the MLMC level
// moments (Sec. II-B, Eq. 9).
#include "mqs_internal.cuh"

namespace mqs {
namespace {

__global__ void k_fill_k0(int32_t* k0, int n, int lps, int steps) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) k0[l] = (l % lps) * steps;
}

// dst(i, l) = src(i, l) for lanes [lane_begin, lane_end), element (i, l) at i*xs + l
__global__ void k_copy_lanes(const double* __restrict__ src, double* __restrict__ dst, int64_t n,
                             int64_t xs, int lb, int le) {
  const int w = le - lb;
  const int64_t total = n * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w;
    const int l = lb + (int)(t % w);
    dst[i * xs + l] = src[i * xs + l];
  }
}

// out[s][i] = lanes[i*xs + s*stride + off]
__global__ void k_to_rows(const double* __restrict__ lanes, int64_t xs, int n, int ns, int stride,
                          int off, double* __restrict__ out) {
  const int64_t total = (int64_t)n * ns;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / n), i = (int)(t % n);
    out[t] = lanes[(int64_t)i * xs + (int64_t)s * stride + off];
  }
}

// lanes[i*xs + s] = rows[s][i]
__global__ void k_from_rows(const double* __restrict__ rows, int n, int ns, double* __restrict__ lanes,
                            int64_t xs) {
  const int64_t total = (int64_t)n * ns;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / ns), s = (int)(t % ns);
    lanes[(int64_t)i * xs + s] = rows[(int64_t)s * n + i];
  }
}

// qoi[s][0] = sf * sum_{j < lps} raw_fine[s*lps + j] (slice order), qoi[s][1] = sc * raw_coarse[s]
__global__ void k_finish_qoi(const double* __restrict__ rf, const double* __restrict__ rc, int ns,
                             int lps, double sf, double sc, double* __restrict__ qoi) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  double acc = 0.0;
  for (int j = 0; j < lps; ++j) acc += rf[(int64_t)s * lps + j];
  qoi[2 * (int64_t)s] = acc * sf;
  qoi[2 * (int64_t)s + 1] = rc ? rc[s] * sc : 0.0;
}

// Pipelined Parareal keeps the per-slice raw QoI partials of iteration k in
// buffer k mod 2 ([2][lanes], lane = sample * M + slice).  Slice s last ran
// its fine propagator in iteration min(K, s + 1): out[l] takes that buffer's
// value.
__global__ void k_gather_qraw(const double* __restrict__ q2, int64_t lanes, int M, int K,
                              double* __restrict__ out) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= lanes) return;
  const int s = (int)(l % M);
  const int k = min(K, s + 1);
  out[l] = q2[(int64_t)(k & 1) * lanes + l];
}

// Neumaier's compensated summation step.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

constexpr int kMomThreads = 256;

// One CTA: Y_s = Q_l - Q_{l-1}; batch mean and sum of squared deviations with
// compensated two-pass sums, merged into the level record {N, mean, M2, 0}
// by the pairwise update n = na + nb, d = mb - ma, mean = ma + d nb / n,
// M2 = M2a + M2b + d^2 na nb / n.
__global__ void k_mlmc_moments(const double* __restrict__ qoi, int ns, double* __restrict__ rec) {
  __shared__ double ss[kMomThreads], sc[kMomThreads];
  __shared__ double mean_b;
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < ns; i += kMomThreads) neumaier(s, c, qoi[2 * i] - qoi[2 * i + 1]);
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, Cc = 0.0;
    for (int t = 0; t < kMomThreads; ++t) {
      neumaier(S, Cc, ss[t]);
      Cc += sc[t];
    }
    mean_b = (S + Cc) / ns;
  }
  __syncthreads();
  const double mb = mean_b;
  s = 0.0;
  c = 0.0;
  for (int i = threadIdx.x; i < ns; i += kMomThreads) {
    const double d = (qoi[2 * i] - qoi[2 * i + 1]) - mb;
    neumaier(s, c, d * d);
  }
  __syncthreads();
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, Cc = 0.0;
    for (int t = 0; t < kMomThreads; ++t) {
      neumaier(S, Cc, ss[t]);
      Cc += sc[t];
    }
    const double m2b = S + Cc;
    const double na = rec[0], ma = rec[1], m2a = rec[2];
    const double nb = (double)ns;
    const double nn = na + nb;
    const double d = mb - ma;
    rec[0] = nn;
    rec[1] = na == 0.0 ? mb : ma + d * (nb / nn);
    rec[2] = na == 0.0 ? m2b : m2a + m2b + d * d * (na * nb / nn);
  }
}

unsigned grid_of(int64_t total, int block) {
  int64_t g = (total + block - 1) / block;
  if (g > 1 << 20) g = 1 << 20;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int fill_k0(int32_t* k0, int n, int lps, int steps, cudaStream_t st) {
  k_fill_k0<<<grid_of(n, 256), 256, 0, st>>>(k0, n, lps, steps);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int copy_lanes(const double* src, double* dst, int64_t n, int64_t xs, int lb, int le, int,
               int, cudaStream_t st) {
  if (le <= lb) return MQS_OK;
  k_copy_lanes<<<grid_of(n * (le - lb), 256), 256, 0, st>>>(src, dst, n, xs, lb, le);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int transpose_to_rows(const double* lanes, int64_t xs, int n, int ns, int stride, int off,
                      double* out, cudaStream_t st) {
  k_to_rows<<<grid_of((int64_t)n * ns, 256), 256, 0, st>>>(lanes, xs, n, ns, stride, off, out);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int transpose_from_rows(const double* rows, int n, int ns, double* lanes, int64_t xs,
                        cudaStream_t st) {
  k_from_rows<<<grid_of((int64_t)n * ns, 256), 256, 0, st>>>(rows, n, ns, lanes, xs);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int finish_qoi(const double* rf, const double* rc, int ns, int lps, double sf, double sc,
               double* qoi, cudaStream_t st) {
  k_finish_qoi<<<grid_of(ns, 128), 128, 0, st>>>(rf, rc, ns, lps, sf, sc, qoi);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int gather_parareal_qraw(const double* q2, int64_t lanes, int M, int K, double* out,
                         cudaStream_t st) {
  k_gather_qraw<<<grid_of(lanes, 128), 128, 0, st>>>(q2, lanes, M, K, out);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int mlmc_accumulate_dev(const double* qoi, int ns, int, double* rec, cudaStream_t st) {
  k_mlmc_moments<<<1, kMomThreads, 0, st>>>(qoi, ns, rec);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

}  // namespace mqs
