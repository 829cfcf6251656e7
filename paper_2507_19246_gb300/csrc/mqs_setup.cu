// Set-up kernels: region reference matrices and load vectors of a mesh
// (Sec. II-A, Eq. 4-5) and per-sample value expansion of M, K and
// A = M/dt + K (Eq. 7) in the batch-fastest layout.
#include "mqs_internal.cuh"

#include <algorithm>
#include <cmath>

namespace mqs {
namespace {

// Area and barycentric gradients of triangle e.  With d = 2 * signed area and
// vertices (x_a, y_a), grad lambda_a = (y_b - y_c, x_c - x_b) / d for the
// cyclic successors b = a+1, c = a+2 (mod 3).
__device__ __forceinline__ void tri_geometry(const double* __restrict__ xy,
                                             const int32_t* __restrict__ tri, int64_t e,
                                             double& area, double gx[3], double gy[3]) {
  double x[3], y[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const int32_t nd = tri[3 * e + v];
    x[v] = xy[2 * (int64_t)nd];
    y[v] = xy[2 * (int64_t)nd + 1];
  }
  const double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    gx[a] = (y[b] - y[c]) / d;
    gy[a] = (x[c] - x[b]) / d;
  }
  area = 0.5 * fabs(d);
}

// One thread per nonzero k: sum the element contributions that land on k,
// split by the triangle's region, in the (sorted) order of the list.
__global__ void k_region_matrices(int64_t nnz, int R, const double* __restrict__ xy,
                                  const int32_t* __restrict__ tri,
                                  const int32_t* __restrict__ region,
                                  const int32_t* __restrict__ cptr,
                                  const int32_t* __restrict__ contrib, double* __restrict__ Mr,
                                  double* __restrict__ Kr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    double m[kMaxRegions], kk[kMaxRegions];
#pragma unroll
    for (int r = 0; r < kMaxRegions; ++r) m[r] = kk[r] = 0.0;
    for (int32_t c = cptr[k]; c < cptr[k + 1]; ++c) {
      const int32_t code = contrib[c];
      const int64_t e = code / 9;
      const int la = (code % 9) / 3, lb = code % 3;
      double area, gx[3], gy[3];
      tri_geometry(xy, tri, e, area, gx, gy);
      const double me = area * (la == lb ? 2.0 : 1.0) / 12.0;     // int N_a N_b
      const double ke = area * (gx[la] * gx[lb] + gy[la] * gy[lb]);  // int grad N_a . grad N_b
      const int r = region[e];
#pragma unroll
      for (int q = 0; q < kMaxRegions; ++q)
        if (q == r) { m[q] += me; kk[q] += ke; }
    }
    for (int r = 0; r < R; ++r) {
      Mr[r * nnz + k] = m[r];
      Kr[r * nnz + k] = kk[r];
    }
  }
}

// One thread per free row i: F_p[i] = sum over source triangles of phase p
// containing the node of coef_T * |T| / 3.
__global__ void k_load_vectors(int n, int P, const double* __restrict__ xy,
                               const int32_t* __restrict__ tri,
                               const int32_t* __restrict__ src_phase,
                               const double* __restrict__ src_coef,
                               const int32_t* __restrict__ lptr,
                               const int32_t* __restrict__ load, double* __restrict__ F) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double f[kMaxPhases] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t c = lptr[i]; c < lptr[i + 1]; ++c) {
      const int64_t e = load[c];
      double area, gx[3], gy[3];
      tri_geometry(xy, tri, e, area, gx, gy);
      const int p = src_phase[e];
#pragma unroll
      for (int q = 0; q < kMaxPhases; ++q)
        if (q == p) f[q] += src_coef[e] * area / 3.0;
    }
    for (int p = 0; p < P; ++p) F[(int64_t)p * n + i] = f[p];
  }
}

// Per-sample values, batch-fastest: element k of sample s at v[k * vs + s].
// A = M/dt + K with M = sum_r sigma_r M_r and K = sum_r nu_r K_r (Eq. 4, 7).
__global__ void k_expand(int64_t nnz, int n_samples, int R, int n_params,
                         const double* __restrict__ params, double dt,
                         const double* __restrict__ Mr, const double* __restrict__ Kr,
                         int64_t vs, double* __restrict__ A, double* __restrict__ M,
                         double* __restrict__ K, float* __restrict__ A32) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= n_samples) return;
  double sig[kMaxRegions], nu[kMaxRegions];
#pragma unroll
  for (int r = 0; r < kMaxRegions; ++r) {
    sig[r] = r < R ? params[(int64_t)s * n_params + r] : 0.0;
    nu[r] = r < R ? params[(int64_t)s * n_params + R + r] : 0.0;
  }
  for (int64_t k = blockIdx.x; k < nnz; k += gridDim.x) {
    double m = 0.0, kk = 0.0;
#pragma unroll
    for (int r = 0; r < kMaxRegions; ++r) {
      if (r < R) {
        m = fma(sig[r], Mr[r * nnz + k], m);
        kk = fma(nu[r], Kr[r * nnz + k], kk);
      }
    }
    const double a = m / dt + kk;
    const int64_t o = k * vs + s;
    if (A) A[o] = a;
    if (M) M[o] = m;
    if (K) K[o] = kk;
    if (A32) A32[o] = (float)a;
  }
}

__global__ void k_inv_diag(int n, int n_samples, const int32_t* __restrict__ diag,
                           const double* __restrict__ A, int64_t vs, double* __restrict__ Dinv,
                           float* __restrict__ Dinv32, int64_t ds) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= n_samples) return;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double d = 1.0 / A[(int64_t)diag[i] * vs + s];
    if (Dinv) Dinv[(int64_t)i * ds + s] = d;
    if (Dinv32) Dinv32[(int64_t)i * ds + s] = (float)d;
  }
}

// lane = sample * lanes_per_sample + j: J0 amp_p and the phase shift phase_p.
__global__ void k_lane_sources(const double* __restrict__ params, int n_samples, int n_params,
                               int R, int P, int lps, double* __restrict__ amp,
                               double* __restrict__ phi) {
  const int lane = blockIdx.x * blockDim.x + threadIdx.x;
  if (lane >= n_samples * lps) return;
  const int s = lane / lps;
  const double* p = params + (int64_t)s * n_params;
  const double j0 = p[2 * R];
  for (int q = 0; q < kMaxPhases; ++q) {
    double a = 0.0, f = 0.0;
    if (q < P) {
      a = j0 * p[2 * R + 1 + q];
      f = p[2 * R + 1 + P + q];
    }
    amp[(int64_t)lane * kMaxPhases + q] = a;
    phi[(int64_t)lane * kMaxPhases + q] = f;
  }
}

// y[s][i] = sum_k vals[k * vs + s] x[s][col_k] (sample-major x, y).
__global__ void k_spmv_rows(int n, int n_samples, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colidx, const double* __restrict__ vals,
                            int64_t vs, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n_samples) return;
  const int s = (int)(t / n), i = (int)(t % n);
  double acc = 0.0;
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
    acc = fma(vals[(int64_t)k * vs + s], x[(int64_t)s * n + colidx[k]], acc);
  y[(int64_t)s * n + i] = acc;
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g > 65535 * 8) g = 65535 * 8;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int assemble_region_matrices(MeshDev& m, const double* xy, const int32_t* tri,
                             const int32_t* region, const int32_t* src_phase,
                             const double* src_coef, const std::vector<int32_t>& contrib_ptr,
                             const std::vector<int32_t>& contrib,
                             const std::vector<int32_t>& load_ptr,
                             const std::vector<int32_t>& load, cudaStream_t st) {
  DevBuf d_xy, d_tri, d_reg, d_ph, d_coef, d_cptr, d_c, d_lptr, d_l;
  const size_t nn = (size_t)m.n_nodes, nt = (size_t)m.n_tri;
  MQS_TRY(d_xy.ensure(nn * 2 * sizeof(double)));
  MQS_TRY(d_tri.ensure(nt * 3 * sizeof(int32_t)));
  MQS_TRY(d_reg.ensure(nt * sizeof(int32_t)));
  MQS_TRY(d_ph.ensure(nt * sizeof(int32_t)));
  MQS_TRY(d_coef.ensure(nt * sizeof(double)));
  MQS_TRY(d_cptr.ensure(contrib_ptr.size() * sizeof(int32_t)));
  MQS_TRY(d_c.ensure(contrib.size() * sizeof(int32_t)));
  MQS_TRY(d_lptr.ensure(load_ptr.size() * sizeof(int32_t)));
  MQS_TRY(d_l.ensure(load.size() * sizeof(int32_t)));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_xy.p, xy, nn * 2 * sizeof(double), cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_tri.p, tri, nt * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_reg.p, region, nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_ph.p, src_phase, nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_coef.p, src_coef, nt * sizeof(double), cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_cptr.p, contrib_ptr.data(), contrib_ptr.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  if (!contrib.empty())
    MQS_CUDA_TRY(cudaMemcpyAsync(d_c.p, contrib.data(), contrib.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
  MQS_CUDA_TRY(cudaMemcpyAsync(d_lptr.p, load_ptr.data(), load_ptr.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  if (!load.empty())
    MQS_CUDA_TRY(cudaMemcpyAsync(d_l.p, load.data(), load.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
  const int R = m.n_regions, P = m.n_phases;
  MQS_TRY(m.Mr.ensure((size_t)R * m.nnz * sizeof(double)));
  MQS_TRY(m.Kr.ensure((size_t)R * m.nnz * sizeof(double)));
  MQS_TRY(m.F.ensure((size_t)(P > 0 ? P : 1) * m.n_free * sizeof(double)));
  k_region_matrices<<<grid_for(m.nnz, 256), 256, 0, st>>>(
      m.nnz, R, d_xy.as<double>(), d_tri.as<int32_t>(), d_reg.as<int32_t>(),
      d_cptr.as<int32_t>(), d_c.as<int32_t>(), m.Mr.as<double>(), m.Kr.as<double>());
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  if (P > 0) {
    k_load_vectors<<<grid_for(m.n_free, 256), 256, 0, st>>>(
        m.n_free, P, d_xy.as<double>(), d_tri.as<int32_t>(), d_ph.as<int32_t>(),
        d_coef.as<double>(), d_lptr.as<int32_t>(), d_l.as<int32_t>(), m.F.as<double>());
    MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  }
  // the temporary buffers are freed when this returns: wait for the kernels
  MQS_CUDA_TRY(cudaStreamSynchronize(st));
  return MQS_OK;
}

int expand_values(const MeshDev& m, const double* params, int n_samples, int n_params,
                  double dt, int64_t vs, double* A, double* M, double* K, float* A32,
                  double* Dinv, float* Dinv32, int64_t ds, cudaStream_t st) {
  const int bx = 64;
  dim3 grid((unsigned)std::min<int64_t>(m.nnz, 4096), (unsigned)((n_samples + bx - 1) / bx));
  k_expand<<<grid, bx, 0, st>>>(m.nnz, n_samples, m.n_regions, n_params, params, dt,
                                m.Mr.as<double>(), m.Kr.as<double>(), vs, A, M, K, A32);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  if (Dinv || Dinv32) {
    dim3 g2((unsigned)std::min(m.n_free, 4096), (unsigned)((n_samples + bx - 1) / bx));
    k_inv_diag<<<g2, bx, 0, st>>>(m.n_free, n_samples, m.diag.as<int32_t>(), A, vs, Dinv,
                                  Dinv32, ds);
    MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  }
  return MQS_OK;
}

int lane_sources(const double* params, int n_samples, int n_params, int n_regions,
                 int n_phases, int lanes_per_sample, double* src_amp, double* src_phi,
                 cudaStream_t st) {
  const int lanes = n_samples * lanes_per_sample;
  k_lane_sources<<<(lanes + 127) / 128, 128, 0, st>>>(params, n_samples, n_params, n_regions,
                                                     n_phases, lanes_per_sample, src_amp,
                                                     src_phi);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

int batched_spmv(const MeshDev& m, const double* vals, int64_t vs, int n_samples,
                 const double* x, double* y, cudaStream_t st) {
  const int64_t work = (int64_t)m.n_free * n_samples;
  k_spmv_rows<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(
      m.n_free, n_samples, m.rowptr.as<int32_t>(), m.colidx.as<int32_t>(), vals, vs, x, y);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

}  // namespace mqs
