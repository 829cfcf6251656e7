// Banded direct solver for the implicit-Euler systems (Sec. II-A, Eq. 7):
// (M/dt + K) is factored once per (sample, dt) by a band Cholesky
// decomposition in a reverse Cuthill-McKee ordering and every step does one
// forward and one backward substitution.
//
// Layout.  A factor is stored by rows: row i holds L(i, i-bw .. i) at
// LB[i*(bw+1) + (c - i + bw)] (entries left of column 0 stay zero); after the
// factorisation every row is scaled to unit diagonal (L~ = D^-1 L), the
// reciprocal diagonal invd[i] = 1 / L(i, i) is kept, and the inverse of each
// 32 x 32 diagonal block of L~ is stored in Binv.  Lane vectors of this solver are
// lane-major ([lane][n]) because one CTA advances one lane.
//
// Kernels.
//  * k_band_fill   scatters the lower-band entries of each sample's A values.
//  * k_band_chol   right-looking band Cholesky, one CTA per factor, in place:
//                  for each column j, L_jj = sqrt(A_jj), scale the column,
//                  rank-1 update of the bw x bw trailing triangle.  Used when
//                  the factors fill the GPU; a few factors go to the cluster
//                  kernel k_band_chol_cl (mqs_cluster.cu), which gives the
//                  same factor bit for bit.
//  * k_direct_propagate  one CTA per lane walks all time steps: right-hand
//                  side (original order) scattered into the permuted work
//                  vector, blocked forward and backward substitution (32-row
//                  blocks: a CTA-wide GEMV against the solved part, then a
//                  warp-level triangular solve of the 32 x 32 diagonal block),
//                  gather back, QoI and y = M a.
//  * k_direct_chain  the Parareal coarse sweep (one CTA per sample) with the
//                  Eq. 12 correction and jump norms fused, lane-major state.
// The two stepping kernels serve the mixed-precision form and FP64 batches
// too large for a shared-memory work vector per lane (256 threads, work
// vector in L2); FP64 stepping with the work vector in shared memory runs
// on the cluster kernels of mqs_cluster.cu.
#include "mqs_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <type_traits>

namespace mqs {
namespace {

constexpr int kDT = 1024;         // threads per CTA
constexpr int kDW = kDT / 32;     // warps per CTA
constexpr int kBlk = 32;          // substitution block (rows)
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA-wide sum (warp butterfly, then warps in order).
template <int NT>
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int j = 0; j < NT / 32; ++j) s += red[j];
  return s;
}

template <typename T>
__global__ void k_band_fill(int64_t nnz, const int32_t* __restrict__ band_idx,
                            const double* __restrict__ A, int64_t vs, int n_fac,
                            int64_t fstride, T* __restrict__ LB) {
  const int64_t total = nnz * n_fac;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / n_fac;
    const int f = (int)(t % n_fac);
    const int32_t b = band_idx[k];
    if (b >= 0) LB[f * fstride + b] = (T)A[k * vs + f];
  }
}

// The products L(i, j) L(k, j) of the trailing updates are summed in a
// separate accumulator S(i, k), which starts at zero, and subtracted from
// A(i, k) once, when column k is factored:
//   L(k, k) = sqrt(A(k, k) - S(k, k)),  L(i, k) = (A(i, k) - S(i, k)) / L(k, k).
// Updating A in place instead rounds every one of the up to bw updates
// against the large running value of A(i, k); on the annulus meshes that made
// a solve about 10-40x less accurate than LAPACK's blocked factorisation,
// while the separate sum is within a few times of it.  S needs only the rows
// of the band window: a ring of bw + 1 rows, row i in slot i mod (bw + 1).
template <typename T>
__global__ void __launch_bounds__(kDT) k_band_chol(T* __restrict__ LBall,
                                                  T* __restrict__ invd_all, int n, int bw,
                                                  int64_t fstride, int32_t* __restrict__ bad,
                                                  T* __restrict__ Sall) {
  extern __shared__ unsigned char colj_raw[];
  T* colj = reinterpret_cast<T*>(colj_raw);   // bw entries of the current column
  __shared__ T s_inv;
  T* LB = LBall + blockIdx.x * fstride;
  T* invd = invd_all + (int64_t)blockIdx.x * n;
  const int W = bw + 1;
  T* S = Sall + (int64_t)blockIdx.x * W * W;
  auto srow = [&](int i) { return S + (int64_t)(i % W) * W; };   // S(i, c) at srow(i)[c - i + bw]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < W * W; t += kDT) S[t] = T(0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    // row j + bw enters the window: its slot held row j - 1, done at column j - 1
    if (j >= 1 && j + bw < n)
      for (int t = threadIdx.x; t < W; t += kDT) srow(j + bw)[t] = T(0);
    if (threadIdx.x == 0) {
      T d = LB[(int64_t)j * W + bw] - srow(j)[bw];
      if (!(d > T(0))) {   // not positive definite: record and continue on a unit pivot
        bad[blockIdx.x] = 1;
        d = T(1);
      }
      d = sqrt(d);
      LB[(int64_t)j * W + bw] = d;
      s_inv = T(1) / d;
      invd[j] = s_inv;
    }
    __syncthreads();
    const T inv = s_inv;
    for (int t = threadIdx.x; t < bw; t += kDT) {
      const int i = j + 1 + t;
      T v = T(0);
      if (i < n) {
        const int64_t o = (int64_t)i * W + (j - i + bw);
        v = (LB[o] - srow(i)[j - i + bw]) * inv;
        LB[o] = v;
      }
      colj[t] = v;
    }
    __syncthreads();
    // S(i, k) += L(i, j) L(k, j) for j < k <= i <= j + bw
    for (int a = warp; a < bw; a += kDW) {
      const int i = j + 1 + a;
      if (i >= n) break;
      const T ca = colj[a];
      if (ca == T(0)) continue;
      T* row = srow(i) + (j + 1 - i + bw);   // column j+1 of row i
      for (int b = lane; b <= a; b += 32) row[b] = fma(ca, colj[b], row[b]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- unit scaling
// After factoring, each row is scaled by its reciprocal diagonal, L~ = D^-1 L
// (unit diagonal), so that L y = b becomes L~ y = D^-1 b and L^T x = y becomes
// L~^T u = y with x = D^-1 u.  The inverse of every 32 x 32 diagonal block of
// L~ is stored as well, which turns the sequential in-block substitution into
// a small dense product.
template <typename T>
__global__ void k_band_unit(T* __restrict__ LBall, const T* __restrict__ invd_all,
                            int n, int bw, int64_t fstride, int n_fac) {
  const int W = bw + 1;
  const int64_t total = (int64_t)n * n_fac;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; t < total;
       t += (int64_t)gridDim.x * blockDim.y) {
    const int f = (int)(t / n), i = (int)(t % n);
    T* row = LBall + f * fstride + (int64_t)i * W;
    const T s = invd_all[(int64_t)f * n + i];
    for (int d = threadIdx.x; d < bw; d += blockDim.x) row[d] *= s;
    if (threadIdx.x == 0) row[bw] = T(1);
  }
}

// One warp per diagonal block: lane c solves L~_blk x = e_c (rows past n are identity).
template <typename T>
__global__ void k_block_inv(const T* __restrict__ LBall, T* __restrict__ Binv_all,
                            int n, int bw, int64_t fstride, int nblk, int n_fac) {
  __shared__ T xs[4][kBlk][kBlk + 1];
  const int wl = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int64_t g = blockIdx.x * 4LL + wl;
  if (g >= (int64_t)nblk * n_fac) return;
  const int f = (int)(g / nblk), blk = (int)(g % nblk);
  const T* LB = LBall + f * fstride;
  T* B = Binv_all + ((int64_t)f * nblk + blk) * kBlk * kBlk;
  const int i0 = blk * kBlk, W = bw + 1;
  for (int r = 0; r < kBlk; ++r) {
    T x = (r == c) ? T(1) : T(0);
    const int i = i0 + r;
    if (i < n) {
      for (int j = 0; j < r; ++j)
        if (r - j <= bw) x = fma(-LB[(int64_t)i * W + (i0 + j - i + bw)], xs[wl][j][c], x);
    }
    xs[wl][r][c] = x;
    __syncwarp();
  }
  for (int r = 0; r < kBlk; ++r) B[r * kBlk + c] = xs[wl][r][c];
}

// ---------------------------------------------------------------- substitution
// Software-pipelined blocked substitution.  While the triangle warp (warp
// Shape<NT>::TRI) finishes block b -- the coupling to the previous block, the
// reduction of the partial sums and the product with the inverted diagonal
// block -- the other warps compute the partial sums of block b+1 against all
// columns solved before block b and stage the 32 x 32 coupling between blocks
// b+1 and b into shared memory.
// NT threads per CTA: warps 0 .. NT/32-2 compute the partial sums, the last
// warp is the triangle warp.
template <int NT>
struct Shape {
  static constexpr int DW = NT / 32;
  static constexpr int TRI = DW - 1;
  static constexpr int GW = DW - 1;
  static_assert(DW >= 2 && DW <= kBlk, "2 to 32 warps");
};

template <typename T>
struct SolveSmem {
  T part[2][kBlk][kBlk + 1];   // [buffer][row][lane] partial sums
  T off[2][kBlk][kBlk + 1];    // [buffer][row][col] coupling block
  T sacc[kBlk];
  double red[32];
};

// L~ y = w in place (w already scaled by D^-1, permuted order).
template <int NT, typename T>
__device__ void forward_subst(const T* __restrict__ LB, const T* __restrict__ Binv,
                              int n, int bw, T* w, SolveSmem<T>& sm) {
  const int W = bw + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (n + kBlk - 1) / kBlk;
  // block 0 has no solved columns: empty partial sums and coupling
  for (int t = threadIdx.x; t < kBlk * (kBlk + 1); t += NT) {
    (&sm.part[0][0][0])[t] = T(0);
    (&sm.off[0][0][0])[t] = T(0);
  }
  __syncthreads();
  for (int b = 0; b < nblk; ++b) {
    const int i0 = b * kBlk, cur = b & 1, nxt = cur ^ 1;
    if (warp == Shape<NT>::TRI) {
      const int i = i0 + lane;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        s0 += sm.part[cur][lane][q];
        s1 += sm.part[cur][lane][q + 1];
        s2 += sm.part[cur][lane][q + 2];
        s3 += sm.part[cur][lane][q + 3];
      }
      if (b > 0) {   // coupling to block b-1 (solved in the previous round)
#pragma unroll
        for (int c = 0; c < kBlk; c += 4) {
          s0 = fma(sm.off[cur][lane][c], w[i0 - kBlk + c], s0);
          s1 = fma(sm.off[cur][lane][c + 1], w[i0 - kBlk + c + 1], s1);
          s2 = fma(sm.off[cur][lane][c + 2], w[i0 - kBlk + c + 2], s2);
          s3 = fma(sm.off[cur][lane][c + 3], w[i0 - kBlk + c + 3], s3);
        }
      }
      sm.sacc[lane] = i < n ? w[i] - ((s0 + s1) + (s2 + s3)) : T(0);
      __syncwarp();
      const T* B = Binv + (int64_t)b * kBlk * kBlk + lane * kBlk;   // row `lane`
      T y0 = T(0), y1 = T(0), y2 = T(0), y3 = T(0);
#pragma unroll
      for (int c = 0; c < kBlk; c += 4) {       // B is zero above the diagonal
        y0 = fma(B[c], sm.sacc[c], y0);
        y1 = fma(B[c + 1], sm.sacc[c + 1], y1);
        y2 = fma(B[c + 2], sm.sacc[c + 2], y2);
        y3 = fma(B[c + 3], sm.sacc[c + 3], y3);
      }
      if (i < n) w[i] = (y0 + y1) + (y2 + y3);
    } else if (b + 1 < nblk) {
      // block b+1 against the columns solved before block b: [i - bw, i0)
      const int j0 = i0 + kBlk;
      for (int r = warp; r < kBlk; r += Shape<NT>::GW) {
        const int i = j0 + r;
        T acc = T(0);
        if (i < n) {
          const T* Lr = LB + (int64_t)i * W + (bw - i);   // Lr[c] = L~(i, c)
          int c = max(0, i - bw) + lane;
          for (; c + 96 < i0; c += 128) {
            const T l0 = Lr[c], l1 = Lr[c + 32], l2 = Lr[c + 64], l3 = Lr[c + 96];
            const T w0 = w[c], w1 = w[c + 32], w2 = w[c + 64], w3 = w[c + 96];
            acc = fma(l0, w0, acc);
            acc = fma(l1, w1, acc);
            acc = fma(l2, w2, acc);
            acc = fma(l3, w3, acc);
          }
          for (; c < i0; c += 32) acc = fma(Lr[c], w[c], acc);
          // coupling L~(i, i0 + lane) to block b, inside the band
          const int col = i0 + lane;
          sm.off[nxt][r][lane] = (i - col <= bw) ? Lr[col] : T(0);
        } else {
          sm.off[nxt][r][lane] = T(0);
        }
        sm.part[nxt][r][lane] = acc;
      }
    }
    __syncthreads();
  }
}

// L~^T u = w in place, from the last block up.
template <int NT, typename T>
__device__ void backward_subst(const T* __restrict__ LB, const T* __restrict__ Binv,
                               int n, int bw, T* w, SolveSmem<T>& sm) {
  const int W = bw + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (n + kBlk - 1) / kBlk;
  for (int t = threadIdx.x; t < kBlk * (kBlk + 1); t += NT) {
    (&sm.part[(nblk - 1) & 1][0][0])[t] = T(0);
    (&sm.off[(nblk - 1) & 1][0][0])[t] = T(0);
  }
  __syncthreads();
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = b * kBlk, cur = b & 1, nxt = cur ^ 1;
    if (warp == Shape<NT>::TRI) {
      const int i = i0 + lane;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
      for (int q = 0; q < 32; q += 4) {        // part[cur][q][col]: q = GEMV slot
        s0 += sm.part[cur][q][lane];
        s1 += sm.part[cur][q + 1][lane];
        s2 += sm.part[cur][q + 2][lane];
        s3 += sm.part[cur][q + 3][lane];
      }
      if (b + 1 < nblk) {   // coupling to block b+1: rows i0+32+c (< n), column i0+lane
        const int kb = i0 + kBlk;
        const int cm = min(kBlk, n - kb);                 // rows of block b+1 that exist
#pragma unroll
        for (int c = 0; c < kBlk; c += 4) {
          if (c < cm) s0 = fma(sm.off[cur][c][lane], w[kb + c], s0);
          if (c + 1 < cm) s1 = fma(sm.off[cur][c + 1][lane], w[kb + c + 1], s1);
          if (c + 2 < cm) s2 = fma(sm.off[cur][c + 2][lane], w[kb + c + 2], s2);
          if (c + 3 < cm) s3 = fma(sm.off[cur][c + 3][lane], w[kb + c + 3], s3);
        }
      }
      sm.sacc[lane] = i < n ? w[i] - ((s0 + s1) + (s2 + s3)) : T(0);
      __syncwarp();
      // u = (L~_blk^-1)^T acc: column `lane` of the inverted block
      const T* B = Binv + (int64_t)b * kBlk * kBlk + lane;
      T u0 = T(0), u1 = T(0), u2 = T(0), u3 = T(0);
#pragma unroll
      for (int c = 0; c < kBlk; c += 4) {       // B is zero above the diagonal
        u0 = fma(B[c * kBlk], sm.sacc[c], u0);
        u1 = fma(B[(c + 1) * kBlk], sm.sacc[c + 1], u1);
        u2 = fma(B[(c + 2) * kBlk], sm.sacc[c + 2], u2);
        u3 = fma(B[(c + 3) * kBlk], sm.sacc[c + 3], u3);
      }
      if (i < n) w[i] = (u0 + u1) + (u2 + u3);
    } else if (b > 0) {
      // block b-1 (columns j0 .. j0+31) against the rows solved before block b:
      // k in [i0 + 32, j0 + 31 + bw]
      const int j0 = i0 - kBlk;
      const int col = j0 + lane;
      T acc = T(0);
      const int kend = min(n - 1, j0 + kBlk - 1 + bw);
      int k = i0 + kBlk + warp;
      for (; k + 3 * Shape<NT>::GW <= kend && k + 3 * Shape<NT>::GW - j0 <= bw; k += 4 * Shape<NT>::GW) {
        const T* r0 = LB + (int64_t)k * W + (col - k + bw);
        const T l0 = r0[0], l1 = r0[Shape<NT>::GW * (W - 1)], l2 = r0[2 * Shape<NT>::GW * (W - 1)],
                     l3 = r0[3 * Shape<NT>::GW * (W - 1)];
        const T w0 = w[k], w1 = w[k + Shape<NT>::GW], w2 = w[k + 2 * Shape<NT>::GW],
                     w3 = w[k + 3 * Shape<NT>::GW];
        acc = fma(l0, w0, acc);
        acc = fma(l1, w1, acc);
        acc = fma(l2, w2, acc);
        acc = fma(l3, w3, acc);
      }
      for (; k <= kend; k += Shape<NT>::GW) {
        const int off = col - k + bw;
        if (off >= 0) acc = fma(LB[(int64_t)k * W + off], w[k], acc);
      }
      sm.part[nxt][warp][lane] = acc;
      if (warp == 0)   // slots without a partial-sum warp
        for (int q = Shape<NT>::GW; q < kBlk; ++q) sm.part[nxt][q][lane] = T(0);
      // coupling rows i0 + r (block b) x column j0 + lane (block b-1)
      for (int r = warp; r < kBlk; r += Shape<NT>::GW) {
        const int kk = i0 + r;
        sm.off[nxt][r][lane] = (kk < n && kk - col <= bw) ? LB[(int64_t)kk * W + (col - kk + bw)] : T(0);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double csr_row(const int32_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ colidx, int i,
                                          const double* __restrict__ vals, int64_t vs,
                                          const double* x) {
  double acc = 0.0;
  for (int k = __ldg(rowptr + i); k < __ldg(rowptr + i + 1); ++k)
    acc = fma(__ldg(vals + (int64_t)k * vs), x[__ldg(colidx + k)], acc);
  return acc;
}

struct DLaneOut {
  double qoi;
};

// Advance one lane by n_steps implicit-Euler steps with the direct solver.
// On return the final state is in a0 (as given).
template <int NT>
__device__ void direct_integrate(const DirectConst& kc, const DirectLane& D, int n_steps,
                                 int64_t k0, SolveSmem<double>& sm, DLaneOut& out) {
  const int n = kc.n;
  double* a0 = D.a0;
  double* a1 = D.a1;
  double* y = D.y;
  extern __shared__ unsigned char dyn_smem[];
  double* w = kc.w_in_smem ? reinterpret_cast<double*>(dyn_smem) : D.w;
  const double* Mv = kc.M + D.vcol;
  const double* Kv = kc.K ? kc.K + D.vcol : nullptr;
  if (D.init_from_a0) {
    for (int i = threadIdx.x; i < n; i += NT) y[i] = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a0);
  } else {
    for (int i = threadIdx.x; i < n; i += NT) {
      a0[i] = 0.0;
      y[i] = 0.0;
    }
  }
  __syncthreads();
  double qacc = 0.0;
  const double dt = D.dt;
  for (int step = 0; step < n_steps; ++step) {
    const double t = D.t0 + (double)(k0 + step + 1) * dt;
    double g[kMaxPhases];
#pragma unroll
    for (int ph = 0; ph < kMaxPhases; ++ph) {
      g[ph] = 0.0;
      if (ph < kc.n_phases) {
        const double arg = kc.omega * t - (2.0 * kPi * ph) / kc.n_phases + D.phase[ph];
        g[ph] = D.amp[ph] * sin(arg);
      }
    }
    for (int i = threadIdx.x; i < n; i += NT) {
      double f = 0.0;
#pragma unroll
      for (int ph = 0; ph < kMaxPhases; ++ph)
        if (ph < kc.n_phases) f = fma(g[ph], __ldg(kc.F + (int64_t)ph * n + i), f);
      const int pi = __ldg(kc.iperm + i);
      w[pi] = (y[i] / dt + f) * D.invd[pi];          // D^-1 b
    }
    __syncthreads();
    forward_subst<NT, double>(D.LB, D.Binv, n, kc.bw, w, sm);
    backward_subst<NT, double>(D.LB, D.Binv, n, kc.bw, w, sm);
    for (int i = threadIdx.x; i < n; i += NT) {
      const int pi = __ldg(kc.iperm + i);
      a1[i] = w[pi] * D.invd[pi];                     // x = D^-1 u
    }
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
      const double yn = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a1);
      if (kc.qoi_kind == MQS_QOI_JOULE) {
        part = fma(a1[i] - a0[i], yn - y[i], part);
      } else {
        part = fma(a1[i], csr_row(kc.rowptr, kc.colidx, i, Kv, kc.vs, a1), part);
      }
      y[i] = yn;
    }
    const double red = block_sum<NT>(part, sm.red);
    qacc += kc.qoi_kind == MQS_QOI_JOULE ? red / dt : 0.5 * red;
    double* tmp = a0;
    a0 = a1;
    a1 = tmp;
    __syncthreads();
  }
  if (n_steps & 1) {
    for (int i = threadIdx.x; i < n; i += NT) a1[i] = a0[i];
    __syncthreads();
  }
  out.qoi = qacc;
}

// Mixed precision: FP32 band factor and FP32 substitutions, refined in FP64.
// Each step starts from x = a_k; every sweep forms the FP64 residual
// r = b - A x with the sample's FP64 matrix values, solves L L^T d = r with
// the FP32 factor and adds d to x in FP64, until ||r|| <= tol ||b|| or the
// sweep limit (status MQS_ST_NOTCONV).
template <int NT>
__device__ void direct_integrate_mixed(const DirectConst& kc, const DirectLane& D, int n_steps,
                                       int64_t k0, SolveSmem<float>& sm, DLaneOut& out) {
  const int n = kc.n;
  double* a0 = D.a0;
  double* a1 = D.a1;
  double* y = D.y;
  double* bvec = D.b;
  extern __shared__ unsigned char dyn_smem[];
  float* w = kc.w_in_smem ? reinterpret_cast<float*>(dyn_smem) : reinterpret_cast<float*>(D.w);
  const double* Mv = kc.M + D.vcol;
  const double* Kv = kc.K ? kc.K + D.vcol : nullptr;
  const double* Av = D.Av;
  if (D.init_from_a0) {
    for (int i = threadIdx.x; i < n; i += NT) y[i] = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a0);
  } else {
    for (int i = threadIdx.x; i < n; i += NT) {
      a0[i] = 0.0;
      y[i] = 0.0;
    }
  }
  __syncthreads();
  double qacc = 0.0;
  int status = 0;
  const double dt = D.dt;
  for (int step = 0; step < n_steps; ++step) {
    const double t = D.t0 + (double)(k0 + step + 1) * dt;
    double g[kMaxPhases];
#pragma unroll
    for (int ph = 0; ph < kMaxPhases; ++ph) {
      g[ph] = 0.0;
      if (ph < kc.n_phases) {
        const double arg = kc.omega * t - (2.0 * kPi * ph) / kc.n_phases + D.phase[ph];
        g[ph] = D.amp[ph] * sin(arg);
      }
    }
    double bb = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
      double f = 0.0;
#pragma unroll
      for (int ph = 0; ph < kMaxPhases; ++ph)
        if (ph < kc.n_phases) f = fma(g[ph], __ldg(kc.F + (int64_t)ph * n + i), f);
      const double bi = y[i] / dt + f;
      bvec[i] = bi;
      a1[i] = a0[i];
      bb = fma(bi, bi, bb);
    }
    bb = block_sum<NT>(bb, sm.red);
    for (int sweep = 0;; ++sweep) {
      double rr = 0.0;
      for (int i = threadIdx.x; i < n; i += NT) {
        const double ri = bvec[i] - csr_row(kc.rowptr, kc.colidx, i, Av, kc.vs, a1);
        rr = fma(ri, ri, rr);
        const int pi = __ldg(kc.iperm + i);
        w[pi] = (float)ri * D.invdf[pi];               // D^-1 r in FP32
      }
      rr = block_sum<NT>(rr, sm.red);                   // also orders the w writes
      if (rr <= kc.tol2 * bb) break;
      if (sweep >= kc.max_sweeps || !isfinite(rr)) {
        status |= isfinite(rr) ? MQS_ST_NOTCONV : MQS_ST_NONFINITE;
        break;
      }
      forward_subst<NT, float>(D.LBf, D.Binvf, n, kc.bw, w, sm);
      backward_subst<NT, float>(D.LBf, D.Binvf, n, kc.bw, w, sm);
      for (int i = threadIdx.x; i < n; i += NT) {
        const int pi = __ldg(kc.iperm + i);
        a1[i] += (double)(w[pi] * D.invdf[pi]);        // x += D^-1 u
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
      const double yn = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a1);
      if (kc.qoi_kind == MQS_QOI_JOULE) {
        part = fma(a1[i] - a0[i], yn - y[i], part);
      } else {
        part = fma(a1[i], csr_row(kc.rowptr, kc.colidx, i, Kv, kc.vs, a1), part);
      }
      y[i] = yn;
    }
    const double red = block_sum<NT>(part, sm.red);
    qacc += kc.qoi_kind == MQS_QOI_JOULE ? red / dt : 0.5 * red;
    double* tmp = a0;
    a0 = a1;
    a1 = tmp;
    __syncthreads();
  }
  if (n_steps & 1) {
    for (int i = threadIdx.x; i < n; i += NT) a1[i] = a0[i];
    __syncthreads();
  }
  out.qoi = qacc;
  if (threadIdx.x == 0 && status && D.status_out) *D.status_out |= status;
}

template <int NT, int PREC>
struct Integrator;
template <int NT>
struct Integrator<NT, 0> {
  using Smem = SolveSmem<double>;
  __device__ static void run(const DirectConst& kc, const DirectLane& D, int n_steps, int64_t k0,
                             Smem& sm, DLaneOut& out) {
    direct_integrate<NT>(kc, D, n_steps, k0, sm, out);
  }
};
template <int NT>
struct Integrator<NT, 1> {
  using Smem = SolveSmem<float>;
  __device__ static void run(const DirectConst& kc, const DirectLane& D, int n_steps, int64_t k0,
                             Smem& sm, DLaneOut& out) {
    direct_integrate_mixed<NT>(kc, D, n_steps, k0, sm, out);
  }
};

template <int NT, int PREC>
__global__ void __launch_bounds__(NT, 1024 / NT) k_direct_propagate(const DirectLane* __restrict__ lanes,
                                                                 DirectConst kc) {
  __shared__ typename Integrator<NT, PREC>::Smem sm;
  const DirectLane D = lanes[blockIdx.x];
  if (D.init_from_a0 && D.a_init) {   // start state held elsewhere: into a0 first
    for (int i = threadIdx.x; i < kc.n; i += NT) D.a0[i] = D.a_init[i];
    __syncthreads();
  }
  DLaneOut out;
  Integrator<NT, PREC>::run(kc, D, D.n_steps, D.k0, sm, out);
  if (threadIdx.x == 0) D.qoi_out[0] = out.qoi * D.qoi_scale;
  if (D.done_flag) {   // results (state, QoI, status) visible before the flag
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(D.done_flag) = 1;
    }
  }
}

// Parareal coarse sweep, one CTA per sample; slice states lane-major
// U/E/G[(sample*M + s) * n + i].
template <int NT, int PREC>
__global__ void __launch_bounds__(NT, 1024 / NT) k_direct_chain(const DirectLane* __restrict__ lanes,
                                                             DirectConst kc, DirectChain ch) {
  __shared__ typename Integrator<NT, PREC>::Smem sm;
  DirectLane D = lanes[blockIdx.x];
  const int n = kc.n;
  const int sample = D.sample;
  D.init_from_a0 = 1;
  const int s_stop = min(ch.s_end, ch.M - 1);
  for (int s = ch.s_begin; s < s_stop; ++s) {
    const int64_t base = ((int64_t)sample * ch.M + s) * n;
    const double* U0 = s == ch.s_first ? ch.U_prev : ch.U_cur;
    for (int i = threadIdx.x; i < n; i += NT) D.a0[i] = U0[base + i];
    __syncthreads();
    DLaneOut out;
    Integrator<NT, PREC>::run(kc, D, ch.steps_per_slice, (int64_t)s * ch.steps_per_slice, sm, out);
    double j2 = 0.0, u2 = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
      const double gn = D.a0[i];
      const double un = ch.first_sweep ? gn : ch.E[base + i] + (gn - ch.G[base + i]);
      const double du = un - ch.U_prev[base + n + i];
      j2 = fma(du, du, j2);
      u2 = fma(un, un, u2);
      ch.U_cur[base + n + i] = un;
      ch.G[base + i] = gn;
    }
    j2 = block_sum<NT>(j2, sm.red);
    u2 = block_sum<NT>(u2, sm.red);
    if (threadIdx.x == 0) {
      ch.jump2[(int64_t)sample * ch.M + s + 1] = j2;
      ch.norm2[(int64_t)sample * ch.M + s + 1] = u2;
    }
    __syncthreads();
  }
}

}  // namespace

int block_count(int n) { return (n + kBlk - 1) / kBlk; }

// Largest n whose work vector fits next to the static shared memory of the
// stepping kernels (227 KB per CTA on sm_103).
int direct_smem_max_n(int mixed) {
  const size_t fixed = mixed ? sizeof(SolveSmem<float>) : sizeof(SolveSmem<double>);
  return (int)((227 * 1024 - fixed - 1024) / (mixed ? sizeof(float) : sizeof(double)));
}

namespace {

int grid_of(int64_t total, int block) {
  int64_t g = (total + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 20));
}

}  // namespace

template <typename T>
int band_factor(const MeshDev& m, const double* A, int64_t vs, int n_fac, T* LB, T* invd, T* Binv,
                int32_t* bad, cudaStream_t st) {
  const int bw = m.bw;
  const int64_t fstride = (int64_t)m.n_free * (bw + 1);
  MQS_CUDA_TRY(cudaMemsetAsync(LB, 0, (size_t)fstride * n_fac * sizeof(T), st));
  MQS_CUDA_TRY(cudaMemsetAsync(bad, 0, (size_t)n_fac * sizeof(int32_t), st));
  k_band_fill<T><<<grid_of(m.nnz * n_fac, 256), 256, 0, st>>>(m.nnz, m.band_idx.as<int32_t>(), A,
                                                            vs, n_fac, fstride, LB);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  int n_sm = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // few factors: each on a cluster of CTAs (env MQS_CHOL_CLUSTER=0/1 forces the choice)
  const char* ev = getenv("MQS_CHOL_CLUSTER");
  const bool few = n_fac * band_chol_cluster_size() <= n_sm;
  const bool use_cluster = ev && *ev ? atoi(ev) != 0 : few;
  if (std::is_same<T, double>::value && use_cluster && band_chol_cluster_fits(bw)) {
    MQS_TRY(band_chol_cluster(reinterpret_cast<double*>(LB), reinterpret_cast<double*>(invd),
                              m.n_free, bw, fstride, n_fac, bad, st));
  } else {
    const size_t smem = (size_t)std::max(bw, 1) * sizeof(T);
    MQS_CUDA_TRY(cudaFuncSetAttribute(k_band_chol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    // accumulator rings, stream-ordered scratch freed behind the kernel
    T* S = nullptr;
    const size_t sbytes = (size_t)n_fac * (bw + 1) * (bw + 1) * sizeof(T);
    MQS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&S), sbytes, st));
    k_band_chol<T><<<n_fac, kDT, smem, st>>>(LB, invd, m.n_free, bw, fstride, bad, S);
    MQS_CUDA_TRY(cudaGetLastError());
    count_launch();
    MQS_CUDA_TRY(cudaFreeAsync(S, st));
  }
  k_band_unit<T><<<grid_of((int64_t)m.n_free * n_fac, 8), dim3(32, 8), 0, st>>>(LB, invd, m.n_free,
                                                                             bw, fstride, n_fac);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  const int nblk = (m.n_free + kBlk - 1) / kBlk;
  k_block_inv<T><<<(unsigned)(((int64_t)nblk * n_fac + 3) / 4), 128, 0, st>>>(
      LB, Binv, m.n_free, bw, fstride, nblk, n_fac);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}
template int band_factor<double>(const MeshDev&, const double*, int64_t, int, double*, double*,
                                 double*, int32_t*, cudaStream_t);
template int band_factor<float>(const MeshDev&, const double*, int64_t, int, float*, float*,
                                float*, int32_t*, cudaStream_t);

size_t direct_smem(const DirectConst& kc) {
  return kc.w_in_smem ? (size_t)kc.n * (kc.mixed ? sizeof(float) : sizeof(double)) : 0;
}

// Threads per lane-CTA: 1024 with the work vector in shared memory (one lane
// per SM) when the lanes do not fill the GPU; 256 with the work vector in L2
// for large batches, so that several lanes per SM overlap their latencies.
int direct_threads(const DirectConst& kc) { return kc.w_in_smem ? 1024 : 256; }

template <int NT, int PREC>
int launch_direct_t(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                    cudaStream_t st) {
  const size_t smem = direct_smem(kc);   // on top of the static SolveSmem
  MQS_CUDA_TRY(cudaFuncSetAttribute(k_direct_propagate<NT, PREC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_direct_propagate<NT, PREC><<<n_lanes, NT, smem, st>>>(d_lanes, kc);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

template <int NT, int PREC>
int launch_chain_t(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                   const DirectChain& ch, cudaStream_t st) {
  const size_t smem = direct_smem(kc);
  MQS_CUDA_TRY(cudaFuncSetAttribute(k_direct_chain<NT, PREC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_direct_chain<NT, PREC><<<n_lanes, NT, smem, st>>>(d_lanes, kc, ch);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

// Lanes the throughput form (256 threads per lane, work vector in L2) keeps
// resident on the whole GPU at once: its CTAs per SM times the SM count.
int direct_lane_slots(int mixed) {
  int dev = 0, n_sm = 0, per_sm = 0;
  MQS_CUDA_TRY(cudaGetDevice(&dev));
  MQS_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const cudaError_t e = mixed
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_direct_propagate<256, 1>, 256, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_direct_propagate<256, 0>, 256, 0);
  if (e != cudaSuccess) {
    set_error("occupancy query failed: %s", cudaGetErrorString(e));
    return -1;
  }
  return per_sm * n_sm;
}

int launch_direct(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc, cudaStream_t st) {
  if (n_lanes <= 0) return MQS_OK;
  if (kc.mixed)
    return direct_threads(kc) == 1024 ? launch_direct_t<1024, 1>(d_lanes, n_lanes, kc, st)
                                      : launch_direct_t<256, 1>(d_lanes, n_lanes, kc, st);
  return direct_threads(kc) == 1024 ? launch_direct_t<1024, 0>(d_lanes, n_lanes, kc, st)
                                    : launch_direct_t<256, 0>(d_lanes, n_lanes, kc, st);
}

int launch_direct_chain(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                        const DirectChain& ch, cudaStream_t st) {
  if (n_lanes <= 0) return MQS_OK;
  if (kc.mixed)
    return direct_threads(kc) == 1024 ? launch_chain_t<1024, 1>(d_lanes, n_lanes, kc, ch, st)
                                      : launch_chain_t<256, 1>(d_lanes, n_lanes, kc, ch, st);
  return direct_threads(kc) == 1024 ? launch_chain_t<1024, 0>(d_lanes, n_lanes, kc, ch, st)
                                    : launch_chain_t<256, 0>(d_lanes, n_lanes, kc, ch, st);
}

}  // namespace mqs
