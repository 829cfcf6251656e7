// Batched implicit-Euler time stepping with a fused per-lane Jacobi-PCG
// (Sec. II-A, Eq. 7) and the Parareal coarse sweep with its fused correction
// and jump norms (Sec. II-C, Eq. 12).
//
// Execution model.  A "tile" is L lanes (samples or Parareal slices) that
// share a step size and a step count.  One thread-block cluster of C CTAs
// (a "team") owns one tile for the whole run: CTA `rank` owns the rows
// [rank*n/C, (rank+1)*n/C) of every lane vector, and the team walks all time
// steps and all CG iterations inside one launch.  Lane vectors are stored
// batch-fastest (element (i, l) at v[i*xs + l]) so that a warp reading one row
// for L lanes issues one contiguous L-wide access; the CSR pattern (rowptr,
// colidx) is shared by all lanes and read once per warp-row.  Per-lane dot
// products are reduced in a fixed order -- thread-serial over rows, warp
// butterfly, warps in order, then the C CTA partials read over distributed
// shared memory in rank order -- so every CTA of the team obtains bitwise the
// same scalars and the result of a lane depends only on the mesh and the
// launch shape (L, C), not on the other lanes of the batch.  Teams never wait
// on each other; cluster barriers are hardware barriers between co-scheduled
// CTAs.
//
// Two arithmetic forms of the CG:
//   PREC = 0 (FP64): Jacobi-PCG entirely in binary64.
//   PREC = 1 (mixed): the matrix values and the search direction used by the
//     SpMV are binary32 (q = A32 * p32 with FP32 accumulation); iterates,
//     residuals and dot products stay binary64, and every `replace_every`
//     iterations -- and before accepting convergence -- the recursive residual
//     is replaced by the true FP64 residual b - A x (iterative refinement
//     without restarting the Krylov recurrence).
#include "mqs_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace mqs {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr double kPi = 3.14159265358979323846;

template <int L>
struct RedSmem {
  double w[3][kWarps][L];   // per-warp partials
  double c[2][3][L];        // per-CTA partials, double-buffered across reductions
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Sum NV per-lane values over all threads of the team holding the same lane.
template <int L, int NV>
__device__ __forceinline__ void team_reduce(double (&v)[NV], RedSmem<L>& sm, int& par,
                                            unsigned C) {
#pragma unroll
  for (int off = L; off < 32; off <<= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  if (wl < L) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sm.w[j][warp][wl] = v[j];
  }
  __syncthreads();
  if (threadIdx.x < L) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += sm.w[j][w][threadIdx.x];
      sm.c[par][j][threadIdx.x] = s;
    }
  }
  cluster_barrier();
  cg::cluster_group cl = cg::this_cluster();
  const int lane = threadIdx.x % L;
  double out[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = 0.0;
  for (unsigned r = 0; r < C; ++r) {
    const double* rem = cl.map_shared_rank(&sm.c[par][0][0], r);
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] += rem[j * L + lane];
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = out[j];
  par ^= 1;
}

// sum_k vals[k*vs] * x[col_k*xs] over row i, k ascending, accumulated in TA.
template <typename TA, typename TV, typename TX>
__device__ __forceinline__ TA row_dot(const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ colidx, int i,
                                      const TV* __restrict__ vals, int64_t vs, const TX* x,
                                      int64_t xs) {
  const int kb = __ldg(rowptr + i), ke = __ldg(rowptr + i + 1);
  TA acc = TA(0);
  for (int k0 = kb; k0 < ke; k0 += 8) {
    int c[8];
    TV v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + j;
      c[j] = k < ke ? __ldg(colidx + k) : 0;
      v[j] = k < ke ? __ldg(vals + (int64_t)k * vs) : TV(0);
    }
    TX xv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xv[j] = (k0 + j < ke) ? x[(int64_t)c[j] * xs] : TX(0);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < ke) acc = fma(TA(v[j]), TA(xv[j]), acc);
  }
  return acc;
}

struct LaneOut {
  double qoi;      // raw QoI sum over the steps of this run
  double iters;    // PCG iterations of this lane
  int status;
};

// Advance the tile `T` by T.n_steps implicit-Euler steps starting at global
// step k0 + k_off of each lane.  On return a0 (as given) holds the final state.
template <int L, int PREC>
__device__ void integrate(const TileDesc& T, const TeamConst& kc, RedSmem<L>& sm, int& par,
                          unsigned rank, unsigned C, int k_off, LaneOut& out) {
  const int lane = threadIdx.x % L;
  const int rslot = threadIdx.x / L;
  constexpr int RP = kThreads / L;
  const int n = kc.n;
  const int r0 = (int)(((int64_t)n * rank) / C);
  const int r1 = (int)(((int64_t)n * (rank + 1)) / C);
  const bool active = lane < T.n_active;
  const int gl = T.lane0 + lane;
  const int64_t xs = T.xs;
  const int64_t vl = (int64_t)lane * T.ls;
  const double* __restrict__ A = T.A + vl;
  const double* __restrict__ Mv = T.M + vl;
  const double* __restrict__ Kv = T.K ? T.K + vl : nullptr;
  const float* __restrict__ A32 = T.A32 ? T.A32 + vl : nullptr;
  const double* __restrict__ Dinv = T.Dinv + vl;
  double* a0 = T.a0 + lane;
  double* a1 = T.a1 + lane;
  double* y = T.y + lane;
  double* r = T.r + lane;
  double* p = T.p + lane;
  double* q = T.q + lane;
  double* z = T.z + lane;
  double* bvec = T.b ? T.b + lane : nullptr;
  float* p32 = T.p32 ? T.p32 + lane : nullptr;
  float* q32 = T.q32 ? T.q32 + lane : nullptr;
  const int32_t* __restrict__ rowptr = kc.rowptr;
  const int32_t* __restrict__ colidx = kc.colidx;

  double amp[kMaxPhases], phase[kMaxPhases];
#pragma unroll
  for (int ph = 0; ph < kMaxPhases; ++ph) {
    amp[ph] = active ? kc.lanes.src_amp[(int64_t)gl * kMaxPhases + ph] : 0.0;
    phase[ph] = active ? kc.lanes.src_phi[(int64_t)gl * kMaxPhases + ph] : 0.0;
  }
  const int64_t k0 = (active ? kc.lanes.k0[gl] : 0) + k_off;

  // initial state and y = M a0
  if (!active) {
    // padded lanes of a tile own no data: they only join the reductions
  } else if (T.init_from_a0) {
    for (int i = r0 + rslot; i < r1; i += RP)
      y[(int64_t)i * xs] = row_dot<double>(rowptr, colidx, i, Mv, T.vs, a0, xs);
  } else {
    for (int i = r0 + rslot; i < r1; i += RP) {
      a0[(int64_t)i * xs] = 0.0;
      y[(int64_t)i * xs] = 0.0;
    }
  }
  cluster_barrier();

  double qacc = 0.0, lane_it = 0.0;
  int status = 0;
  const double dt = T.dt;
  for (int step = 0; step < T.n_steps; ++step) {
    // source r(t_{k+1}) of Eq. 5 for this lane
    const double t = T.t0 + (double)(k0 + step + 1) * dt;
    double g[kMaxPhases];
#pragma unroll
    for (int ph = 0; ph < kMaxPhases; ++ph) {
      g[ph] = 0.0;
      if (ph < kc.n_phases) {
        const double arg = kc.omega * t - (2.0 * kPi * ph) / kc.n_phases + phase[ph];
        g[ph] = amp[ph] * sin(arg);
      }
    }
    // RHS (Eq. 7): b = (M a_k)/dt + r(t_{k+1}); warm start x = a_k; r = b - A x
    double red3[3] = {0.0, 0.0, 0.0};
    for (int i = r0 + rslot; active && i < r1; i += RP) {
      const int64_t o = (int64_t)i * xs;
      double f = 0.0;
#pragma unroll
      for (int ph = 0; ph < kMaxPhases; ++ph)
        if (ph < kc.n_phases) f = fma(g[ph], __ldg(kc.F + (int64_t)ph * n + i), f);
      const double bi = y[o] / dt + f;
      const double ax = row_dot<double>(rowptr, colidx, i, A, T.vs, a0, xs);
      const double ri = bi - ax;
      const double zi = Dinv[(int64_t)i * T.ds] * ri;
      a1[o] = a0[o];
      r[o] = ri;
      p[o] = zi;
      if (PREC == 1) {
        bvec[o] = bi;
        p32[o] = (float)zi;
      }
      red3[0] = fma(ri, zi, red3[0]);
      red3[1] = fma(ri, ri, red3[1]);
      red3[2] = fma(bi, bi, red3[2]);
    }
    team_reduce<L, 3>(red3, sm, par, C);
    double rz = red3[0], rr = red3[1];
    const double bb = red3[2];
    const double thr = kc.tol2 * bb;
    bool conv = !active || rr <= thr;
    if (active && !(isfinite(rr) && isfinite(bb))) {
      status |= MQS_ST_NONFINITE;
      conv = true;
    }
    int it = 0;
    while (!__all_sync(0xffffffffu, conv) && it < kc.max_it) {
      // S: q = A p and (p, q)
      double red1[1] = {0.0};
      if (!conv) {
        for (int i = r0 + rslot; i < r1; i += RP) {
          const int64_t o = (int64_t)i * xs;
          double qi;
          if (PREC == 0) {
            qi = row_dot<double>(rowptr, colidx, i, A, T.vs, p, xs);
            q[o] = qi;
          } else {
            const float qf = row_dot<float>(rowptr, colidx, i, A32, T.vs, p32, xs);
            q32[o] = qf;
            qi = (double)qf;
          }
          red1[0] = fma(p[o], qi, red1[0]);
        }
      }
      team_reduce<L, 1>(red1, sm, par, C);
      const double alpha = conv ? 0.0 : rz / red1[0];
      // U: x += alpha p, r -= alpha q, z = D^-1 r, (r, z), (r, r)
      double red2[2] = {0.0, 0.0};
      if (!conv) {
        for (int i = r0 + rslot; i < r1; i += RP) {
          const int64_t o = (int64_t)i * xs;
          const double qi = PREC == 0 ? q[o] : (double)q32[o];
          a1[o] = fma(alpha, p[o], a1[o]);
          const double ri = fma(-alpha, qi, r[o]);
          const double zi = Dinv[(int64_t)i * T.ds] * ri;
          r[o] = ri;
          z[o] = zi;
          red2[0] = fma(ri, zi, red2[0]);
          red2[1] = fma(ri, ri, red2[1]);
        }
      }
      team_reduce<L, 2>(red2, sm, par, C);
      double rz_new = red2[0], rr_new = red2[1];
      bool conv_next = conv || rr_new <= thr;
      if (PREC == 1) {
        // FP64 residual replacement: periodically and before accepting convergence
        const bool periodic = ((it + 1) % kc.replace_every) == 0;
        const bool want = !conv && (periodic || conv_next);
        if (__any_sync(0xffffffffu, want)) {
          double red2b[2] = {0.0, 0.0};
          if (!conv) {
            for (int i = r0 + rslot; i < r1; i += RP) {
              const int64_t o = (int64_t)i * xs;
              const double ax = row_dot<double>(rowptr, colidx, i, A, T.vs, a1, xs);
              const double ri = bvec[o] - ax;
              const double zi = Dinv[(int64_t)i * T.ds] * ri;
              r[o] = ri;
              z[o] = zi;
              red2b[0] = fma(ri, zi, red2b[0]);
              red2b[1] = fma(ri, ri, red2b[1]);
            }
          }
          team_reduce<L, 2>(red2b, sm, par, C);
          rz_new = red2b[0];
          rr_new = red2b[1];
          conv_next = conv || rr_new <= thr;
        }
      }
      if (!conv) {
        if (!isfinite(rr_new)) {
          status |= MQS_ST_NONFINITE;
          conv_next = true;
        }
        const double beta = rz_new / rz;
        rz = rz_new;
        rr = rr_new;
        lane_it += 1.0;
        if (!conv_next) {
          // P: p = z + beta p
          for (int i = r0 + rslot; i < r1; i += RP) {
            const int64_t o = (int64_t)i * xs;
            const double pi = fma(beta, p[o], z[o]);
            p[o] = pi;
            if (PREC == 1) p32[o] = (float)pi;
          }
        }
      }
      cluster_barrier();
      conv = conv_next;
      ++it;
    }
    if (!conv) status |= MQS_ST_NOTCONV;
    // QoI (Eq. 26 / energy) and y_{k+1} = M a_{k+1}
    double redq[1] = {0.0};
    for (int i = r0 + rslot; active && i < r1; i += RP) {
      const int64_t o = (int64_t)i * xs;
      const double yn = row_dot<double>(rowptr, colidx, i, Mv, T.vs, a1, xs);
      if (kc.qoi_kind == MQS_QOI_JOULE) {
        redq[0] = fma(a1[o] - a0[o], yn - y[o], redq[0]);
      } else {
        const double ka = row_dot<double>(rowptr, colidx, i, Kv, T.vs, a1, xs);
        redq[0] = fma(a1[o], ka, redq[0]);
      }
      y[o] = yn;
    }
    team_reduce<L, 1>(redq, sm, par, C);
    if (kc.qoi_kind == MQS_QOI_JOULE)
      qacc += redq[0] / dt;
    else
      qacc += 0.5 * redq[0];
    double* tmp = a0;
    a0 = a1;
    a1 = tmp;
  }
  if (T.n_steps & 1) {
    // the latest state is in the a1 buffer: copy it back to the a0 buffer
    for (int i = r0 + rslot; active && i < r1; i += RP) a1[(int64_t)i * xs] = a0[(int64_t)i * xs];
    cluster_barrier();
  }
  out.qoi = qacc;
  out.iters = lane_it;
  out.status = status;
}

template <int L, int PREC>
__global__ void __launch_bounds__(kThreads) k_propagate(const TileDesc* __restrict__ tiles,
                                                        TeamConst kc) {
  __shared__ RedSmem<L> sm;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned C = cl.num_blocks(), rank = cl.block_rank();
  const TileDesc T = tiles[blockIdx.x / C];
  int par = 0;
  LaneOut out;
  integrate<L, PREC>(T, kc, sm, par, rank, C, 0, out);
  const int lane = threadIdx.x % L;
  if (rank == 0 && threadIdx.x < L && lane < T.n_active) {
    const int gl = T.lane0 + lane;
    kc.lanes.qoi_raw[gl] = out.qoi;
    kc.lanes.iters[gl] += out.iters;
    kc.lanes.status[gl] |= out.status;
  }
}

// Parareal coarse sweep for one tile of chain lanes (one lane per sample):
// for s = s_begin .. M-2, propagate U[s] over slice s with the coarse step and
// apply Eq. 12's update U[s+1] = E[s] + (G_new - G_old[s]) (first sweep:
// U[s+1] = G_new), with the per-slice squared jump and norm.
template <int L, int PREC>
__global__ void __launch_bounds__(kThreads) k_chain(const TileDesc* __restrict__ tiles,
                                                    TeamConst kc, ChainDesc ch) {
  __shared__ RedSmem<L> sm;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned C = cl.num_blocks(), rank = cl.block_rank();
  TileDesc T = tiles[blockIdx.x / C];
  const int lane = threadIdx.x % L;
  const int rslot = threadIdx.x / L;
  constexpr int RP = kThreads / L;
  const int n = kc.n;
  const int r0 = (int)(((int64_t)n * rank) / C);
  const int r1 = (int)(((int64_t)n * (rank + 1)) / C);
  const bool active = lane < T.n_active;
  const int sample = T.lane0 + lane;           // chain lane == sample index
  int par = 0;
  double it_sum = 0.0;
  int st_sum = 0;
  T.init_from_a0 = 1;
  T.n_steps = ch.steps_per_slice;
  for (int s = ch.s_begin; s < ch.M - 1; ++s) {
    const int64_t col = (int64_t)sample * ch.M + s;
    for (int i = r0 + rslot; i < r1; i += RP)
      if (active) T.a0[(int64_t)i * T.xs + lane] = ch.U[(int64_t)i * ch.xs_par + col];
    cluster_barrier();
    LaneOut out;
    integrate<L, PREC>(T, kc, sm, par, rank, C, s * ch.steps_per_slice, out);
    it_sum += out.iters;
    st_sum |= out.status;
    double red[2] = {0.0, 0.0};
    for (int i = r0 + rslot; i < r1; i += RP) {
      if (!active) continue;
      const double gn = T.a0[(int64_t)i * T.xs + lane];
      const int64_t o = (int64_t)i * ch.xs_par + col;
      double un;
      if (ch.first_sweep) {
        un = gn;
      } else {
        un = ch.E[o] + (gn - ch.G[o]);
      }
      const double du = un - ch.U[o + 1];
      red[0] = fma(du, du, red[0]);
      red[1] = fma(un, un, red[1]);
      ch.U[o + 1] = un;
      ch.G[o] = gn;
    }
    team_reduce<L, 2>(red, sm, par, C);
    if (rank == 0 && threadIdx.x < L && active) {
      ch.jump2[(int64_t)sample * ch.M + s + 1] = red[0];
      ch.norm2[(int64_t)sample * ch.M + s + 1] = red[1];
    }
  }
  if (rank == 0 && threadIdx.x < L && active) {
    const int gl = T.lane0 + lane;
    kc.lanes.iters[gl] += it_sum;
    kc.lanes.status[gl] |= st_sum;
  }
}

template <int L, int PREC>
int launch_prop_t(const TileDesc* d_tiles, int n_tiles, int C, const TeamConst& kc,
                  cudaStream_t st) {
  auto kern = k_propagate<L, PREC>;
  if (C > 8) MQS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_tiles * C));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MQS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, d_tiles, kc));
  count_launch();
  return MQS_OK;
}

template <int L, int PREC>
int launch_chain_t(const TileDesc* d_tiles, int n_tiles, int C, const TeamConst& kc,
                   const ChainDesc& ch, cudaStream_t st) {
  auto kern = k_chain<L, PREC>;
  if (C > 8) MQS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_tiles * C));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MQS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, d_tiles, kc, ch));
  count_launch();
  return MQS_OK;
}

template <class K>
int active_clusters(K kern, int C) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * 2));
  cfg.blockDim = dim3(kThreads);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int num = 0;
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                   cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveClusters(&num, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

template <int L, int PREC>
int active_t(int C) {
  return std::min(active_clusters(k_propagate<L, PREC>, C), active_clusters(k_chain<L, PREC>, C));
}

template <int L, int PREC>
int max_cluster_t() {
  for (int C = 16; C > 1; C /= 2)
    if (active_t<L, PREC>(C) > 0) return C;
  return 1;
}

}  // namespace

int team_threads() { return kThreads; }

// Number of clusters of size C of the team kernels that can be resident at once.
int max_active_clusters(int L, int precision, int C) {
  static int cache[6][2][17] = {};
  int li = 0;
  while ((1 << li) < L && li < 5) ++li;
  const int pi = precision ? 1 : 0;
  if (C < 1 || C > 16) return 0;
  if (cache[li][pi][C] == 0) {
    int v = 0;
    switch (L) {
      case 1: v = pi ? active_t<1, 1>(C) : active_t<1, 0>(C); break;
      case 2: v = pi ? active_t<2, 1>(C) : active_t<2, 0>(C); break;
      case 4: v = pi ? active_t<4, 1>(C) : active_t<4, 0>(C); break;
      case 8: v = pi ? active_t<8, 1>(C) : active_t<8, 0>(C); break;
      case 16: v = pi ? active_t<16, 1>(C) : active_t<16, 0>(C); break;
      default: v = pi ? active_t<32, 1>(C) : active_t<32, 0>(C); break;
    }
    cache[li][pi][C] = v > 0 ? v : -1;
  }
  return cache[li][pi][C] > 0 ? cache[li][pi][C] : 0;
}

// Largest cluster size (16, 8, 4, 2 or 1) both team kernels of this tile
// width and precision can be launched with; cached per (L, precision).
int max_cluster(int L, int precision, int) {
  static int cache[6][2] = {};
  int li = 0;
  while ((1 << li) < L && li < 5) ++li;
  const int pi = precision ? 1 : 0;
  if (cache[li][pi] == 0) {
    int c = 1;
    switch (L) {
      case 1: c = pi ? max_cluster_t<1, 1>() : max_cluster_t<1, 0>(); break;
      case 2: c = pi ? max_cluster_t<2, 1>() : max_cluster_t<2, 0>(); break;
      case 4: c = pi ? max_cluster_t<4, 1>() : max_cluster_t<4, 0>(); break;
      case 8: c = pi ? max_cluster_t<8, 1>() : max_cluster_t<8, 0>(); break;
      case 16: c = pi ? max_cluster_t<16, 1>() : max_cluster_t<16, 0>(); break;
      default: c = pi ? max_cluster_t<32, 1>() : max_cluster_t<32, 0>(); break;
    }
    cache[li][pi] = c;
  }
  return cache[li][pi];
}

#define MQS_DISPATCH_L(FN, ...)                                               \
  switch (L) {                                                                \
    case 1: return precision ? FN<1, 1>(__VA_ARGS__) : FN<1, 0>(__VA_ARGS__); \
    case 2: return precision ? FN<2, 1>(__VA_ARGS__) : FN<2, 0>(__VA_ARGS__); \
    case 4: return precision ? FN<4, 1>(__VA_ARGS__) : FN<4, 0>(__VA_ARGS__); \
    case 8: return precision ? FN<8, 1>(__VA_ARGS__) : FN<8, 0>(__VA_ARGS__); \
    case 16: return precision ? FN<16, 1>(__VA_ARGS__) : FN<16, 0>(__VA_ARGS__); \
    case 32: return precision ? FN<32, 1>(__VA_ARGS__) : FN<32, 0>(__VA_ARGS__); \
    default: set_error("unsupported lane tile width %d", L); return MQS_EINVAL; \
  }

int launch_propagate(const TileDesc* d_tiles, int n_tiles, int L, int C, int precision,
                     const TeamConst& kc, cudaStream_t st) {
  if (n_tiles <= 0) return MQS_OK;
  if (C < 1 || C > 16) {
    set_error("cluster size %d out of range", C);
    return MQS_EINVAL;
  }
  MQS_DISPATCH_L(launch_prop_t, d_tiles, n_tiles, C, kc, st)
}

int launch_chain(const TileDesc* d_tiles, int n_tiles, int L, int C, int precision,
                 const TeamConst& kc, const ChainDesc& ch, cudaStream_t st) {
  if (n_tiles <= 0) return MQS_OK;
  if (C < 1 || C > 16) {
    set_error("cluster size %d out of range", C);
    return MQS_EINVAL;
  }
  MQS_DISPATCH_L(launch_chain_t, d_tiles, n_tiles, C, kc, ch, st)
}

}  // namespace mqs
