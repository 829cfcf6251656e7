// Banded direct solver, FP64 stepping kernels with the block substitution
// spread over warps and, optionally, over the CTAs of a thread-block cluster
// (Sec. II-A, Eq. 7: one factorisation per (sample, dt), one forward and one
// backward substitution per implicit-Euler step).
//
// FP64 on this GPU retires one warp instruction per 64 cycles on each of the
// four SM sub-partitions, whatever the number of active lanes, and a dependent
// FP64 instruction waits as long.  The substitution is therefore organised so
// that (1) the dense work of every 64-row block runs on several warps
// instead of one, (2) the band products (GEMV) run on other
// warps with long per-lane FMA chains and few reduction levels, and (3) one
// lane may be split over a cluster of CL CTAs on CL SMs.
//
// Algebra (unit lower factor L~ = D^-1 L, 64-row blocks, B_b = L~_bb^-1):
//   forward  L~ y = w:    y_b = B_b (w_b - P_b) - C1_b y_{b-1} - C2_b y_{b-2},
//                         C1_b = B_b L~_{b,b-1}, C2_b = B_b L~_{b,b-2},
//                         P_b = sum_{k <= b-3} L~_bk y_k
//   backward L~^T u = y:  u_b = B_b^T (y_b - Q_b) - D1_b u_{b+1} - D2_b u_{b+2},
//                         D1_b = B_b^T L~_{b+1,b}^T, D2_b = B_b^T L~_{b+2,b}^T,
//                         Q_b = sum_{k >= b+3} L~_kb^T u_k
// The couplings are precomputed with the factor, laid out so that every warp
// load is coalesced.  Warp roles: GEMV warps form s_b = w_b - P_b (or y_b -
// Q_b) for the block solved two rounds later; pre warps form pre_b = B_b s_b -
// C2_b y_{b-2} one round ahead (B_b s_b as soon as s_b is ready, the C2 term
// once the exchange warps have their C1 products, skipping the zero products
// of the triangular B_b); exchange warps gather the last block, form
// v_b = pre_b - C1_b y_{b-1} and send it, which is the whole critical path of
// a round, kept as far as possible alone on the FP64 pipe.  The warp groups
// hand data over through release/acquire progress counters in shared memory,
// never through a CTA-wide barrier.
//
// Cluster split: every CTA keeps the permuted work vector in shared memory --
// a full copy where it fits, otherwise its own rows and a ring of recently
// solved rows -- and owns rows q*R .. q*R+R-1 (R = 64/CL) of every block, in
// the band ordering.  Per block it computes s for its own rows and its share
// of the block solve, v_q = pre_q - C1_b[:, own] y_{b-1}[own], which it sends
// to every CTA of the cluster with asynchronous DSMEM stores that complete on
// the receiver's mbarrier (no fence on the sending side, no cluster barrier
// per block); each CTA adds the CL shares in rank order, so all copies (full
// or ring) hold identical values.  Waits are bounded: a wait that runs out
// sets MQS_ST_TIMEOUT on the lane and the kernel skips every later wait.
// Node-wise work (right-hand side, y = M a, QoI) is split by the same row
// ownership, so a step exchanges no data through global memory except the new
// state a1, which is published by a cluster barrier before y = M a1.
#include "mqs_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

namespace mqs {
namespace {

namespace cg = cooperative_groups;

constexpr int kB = 64;       // rows per substitution block (one exchange round per block)
constexpr int kNT = 512;     // threads per CTA
constexpr int kNW = kNT / 32;
constexpr int kPF = 24;      // values prefetched per lane (registers)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWaitLimit = 1 << 20;   // mbarrier polls before a wait gives up
constexpr int kSpinLimit = 1 << 24;   // progress-counter polls before a wait gives up
// bytes of block-solve shares a CTA receives from the other CTAs per round
template <int CL>
constexpr uint32_t kShareTx = (CL - 1) * kB * sizeof(double);
constexpr double kPi = 3.14159265358979323846;

// Warp roles per cluster size (R = 64/CL own rows per block):
//  * exchange warps X (gather, v = pre - C1 y, send) and pre warps P, each
//    group covering the 64 rows of a block with RW rows per warp and
//    LPR = 32/RW lanes per row (own rows t = g + LPR k of a lane; the P group
//    is wider with 2 CTAs so that a lane's operands fit in registers);
//  * GEMV warps: forward items of 4 lanes (own row t, chunk h), H chunks
//    per row inside one warp; backward TB own columns per warp, KG = 32/TB
//    row groups.
// With 8 CTAs the exchange warps sit alone on sub-partitions 0 and 1, the pre
// and GEMV warps share 2 and 3.
template <int CL>
struct Split {
  static constexpr int R = kB / CL;
  static constexpr int NX = CL == 8 ? 2 : 4;            // exchange warps
  static constexpr int NP = CL == 2 ? 8 : NX;           // pre warps
  static constexpr int RW = kB / NX, LPR = 32 / RW;     // exchange: rows per warp, lanes per row
  static constexpr int RWP = kB / NP, LPRP = 32 / RWP;  // pre: rows per warp, lanes per row
  static constexpr int X0 = 0, P0 = NX;                 // first exchange / pre warp
  static constexpr int GW = CL == 1 ? 8 : (CL == 8 ? 2 : 4);   // GEMV warps
  static constexpr int GW0 = CL == 8 ? 6 : NX + NP;     // first GEMV warp
  static constexpr int H = 8 * GW / R;                  // forward chunks per own row
  static constexpr int TB = R / GW;                     // backward own columns per GEMV warp
  static constexpr int KG = 32 / TB;                    // backward row groups per own column
  static constexpr int TPX = R / LPR;                   // own rows per exchange lane
  static constexpr int TPP = R / LPRP;                  // own rows per pre lane
  static constexpr bool PF_X = TPX <= kPF;              // exchange lanes prefetch C1
  static constexpr bool PF_B = TPP <= kPF;              // pre lanes prefetch B
  static constexpr bool PF_C2 = 2 * TPP <= kPF;         // ... and C2
  static_assert(R * H == 8 * GW && H >= 1 && H <= 8, "forward items fill the GEMV warps");
  static_assert(TB >= 1 && TB * GW == R && KG >= 1, "backward columns fill the GEMV warps");
  static_assert(RW * LPR == 32 && R % LPR == 0 && RWP * LPRP == 32 && R % LPRP == 0, "lanes");
  static_assert(P0 >= X0 + NX && GW0 >= P0 + NP && GW0 + GW <= kNW, "disjoint warp roles");
};

template <int CL>
struct CSmem {
  double V[2][CL][kB];                       // block-solve shares [round parity][rank][row]
  double s[4][Split<CL>::R];                 // own rows' s of the block solves, ring by round
  double pre[2][kB];                         // pre of the block solves, by round parity
  unsigned long long mbar[2];                // share arrivals of V[0], V[1]
  int ydone;                                 // rounds whose solved block is in the copy
  int sdone;                                 // rounds whose s is in the ring
  int pdone;                                 // rounds whose pre is in shared memory
  int ccount;                                // exchange warps done with their C1 product
  int err;                                   // a wait ran out
  int flag_pub[2];                           // step-boundary snapshot: 1 error, 2 cancelled
  double red[kNW];
  double cred[CL][2];                        // per-rank partial sums for cluster reductions
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// 8-byte store into another CTA's shared memory that completes (bytes) on
// that CTA's mbarrier.
__device__ __forceinline__ void st_async(uint32_t raddr, double v, uint32_t rmbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
               :: "r"(raddr), "d"(v), "r"(rmbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar) : "memory");
}

// The single arrival of a phase, announcing tx bytes.
__device__ __forceinline__ void mbar_arm(uint32_t mbar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(tx)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity, at most kWaitLimit polls; after a
// failed wait every later wait of the CTA returns at once.
__device__ __forceinline__ void mbar_wait(uint32_t mbar, uint32_t parity, int* err) {
  if (*reinterpret_cast<volatile int*>(err)) return;
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(mbar, parity)) return;
  *reinterpret_cast<volatile int*>(err) = 1;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.cta.shared.s32 [%0], %1;" :: "r"(smem_addr(p)), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}

// Wait until a progress counter reaches target, at most kSpinLimit polls.
// The hand-offs inside a CTA take microseconds, so the wait spins (a sleep
// between polls costs far more than it saves).
__device__ __forceinline__ void wait_count(const int* p, int target, int* err) {
  if (*reinterpret_cast<volatile int*>(err)) return;
  for (int it = 0; it < kSpinLimit; ++it)
    if (ld_acquire(p) >= target) return;
  *reinterpret_cast<volatile int*>(err) = 1;
}

// Barrier of one warp group (ids 1, 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Deterministic CTA-wide sum (warp butterfly, then warps in order).
__device__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int j = 0; j < kNW; ++j) s += red[j];
  return s;
}

// Sum of a per-CTA value over the cluster, in rank order (identical on every
// rank).  slot selects one of two independent sums.
template <int CL>
__device__ double cluster_sum(double v, CSmem<CL>& sm, int slot, unsigned q) {
  if constexpr (CL == 1) {
    return v;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < CL) *cl.map_shared_rank(&sm.cred[q][slot], threadIdx.x) = v;
    cluster_sync_all();
    double s = 0.0;
    for (int p = 0; p < CL; ++p) s += sm.cred[p][slot];
    cluster_sync_all();   // slots free for the next use
    return s;
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

// Rows of the solved-row ring: a power of two of at least bw + 256.  While
// the band products of round j read rows down to (first row of block j) - bw,
// the exchange warps can have stored at most the blocks up to j - 1 (they
// wait for round j's pre values, which need round j's band products): a span
// of bw + 64 rows, so bw + 256 leaves slack.
__host__ __device__ inline int cluster_ring_rows(int bw) {
  int r = 256;
  while (r < bw + 4 * 64) r <<= 1;
  return r;
}

// Own rows per CTA: R = 64/CL of each 64-row block.
template <int CL>
__host__ __device__ inline int own_rows(int n) {
  return ((n + 63) / 64) * (64 / CL);
}

// One GEMV work item of a lane: cnt band values at LB[off + j*step], each
// multiplied by w[w0 + j*wstep].
struct GemvDesc {
  int64_t off, step;
  int cnt, w0, wstep;
};

// ---------------------------------------------------------------- substitution
// FULL: every CTA keeps the whole permuted work vector (own = ring = w,
// indexed by row) -- the layout when n doubles fit a CTA's shared memory;
// otherwise own rows plus the ring of solved rows (below).  The arithmetic and
// its order are the same in both.
template <int CL, bool FULL>
struct Subst {
  using S = Split<CL>;
  static constexpr int kBB = kB * kB;
  const double* __restrict__ LB;
  const double* __restrict__ B;    // 64 x 64 diagonal-block inverses [b][r][t]
  const double* __restrict__ BT;   // B^T: [b][t][r]
  const double* __restrict__ C1;   // [b][t][r]
  const double* __restrict__ C2;   // [b][t][r]
  const double* __restrict__ D1;   // D1_b^T: [b][t][r]
  const double* __restrict__ D2;   // D2_b^T: [b][t][r]
  // work vector: this CTA's own rows of every block (own[b * R + t] = row
  // b*64 + q*R + t) and a ring of the most recently solved rows of all CTAs
  // (row r at ring[r & ring_mask]); band products read only rows within the
  // bandwidth of the block being solved, so the ring holds them
  double* own;
  double* ring;
  int ring_mask;
  CSmem<CL>& sm;
  int n, bw, W, nblk, q;
  // lane roles
  int warp, lane;
  int f_t, f_h, f_g;     // forward GEMV item: own row, chunk, lane in chunk
  int b_t, b_kg, gw;     // backward GEMV: own column, row group; GEMV warp index
  int x_r, x_g;          // exchange lane: block row, term group (own rows t = x_g + LPR k)
  int p_r, p_g;          // pre lane: block row, term group (own rows t = p_g + LPRP k)
  int64_t rounds = 0;    // substitution rounds completed (sets the mbarrier phase parity)
  bool stall = false;    // test hook (one-CTA form): the first wait is on a count nothing reaches

  __device__ Subst(const DirectLane& D, double* own_, double* ring_, int ring_rows,
                   CSmem<CL>& sm_, int n_, int bw_, int q_)
      : LB(D.LB), B(D.B64), BT(D.B64T), C1(D.C1), C2(D.C2), D1(D.D1), D2(D.D2), own(own_), ring(ring_),
        ring_mask(ring_rows - 1), sm(sm_), n(n_), bw(bw_), W(bw_ + 1),
        nblk((n_ + kB - 1) / kB), q(q_) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    gw = warp - S::GW0;
    const int item = gw * 8 + (lane >> 2);
    f_t = item / S::H;
    f_h = item % S::H;
    f_g = lane & 3;
    b_t = gw * S::TB + lane % S::TB;
    b_kg = lane / S::TB;
    x_r = (warp - S::X0) * S::RW + lane % S::RW;
    x_g = lane / S::RW;
    p_r = (warp - S::P0) * S::RWP + lane % S::RWP;
    p_g = lane / S::RWP;
  }

  __device__ bool is_exch() const { return warp >= S::X0 && warp < S::X0 + S::NX; }
  __device__ bool is_pre() const { return warp >= S::P0 && warp < S::P0 + S::NP; }
  __device__ bool is_gemv() const { return warp >= S::GW0 && warp < S::GW0 + S::GW; }
  __device__ int block_of(int g) const { return g < nblk ? g : 2 * nblk - 1 - g; }
  // storage of own row t of block blk
  __device__ double& own_at(int blk, int t) const {
    return FULL ? own[blk * kB + q * S::R + t] : own[blk * S::R + t];
  }
  // own row t of block blk (0 past n)
  __device__ double own_val(int blk, int t) const {
    const int row = blk * kB + q * S::R + t;
    return row < n ? own_at(blk, t) : 0.0;
  }
  // storage index of own node idx (row pi) in the node-wise phases
  __device__ int own_index(int idx, int pi) const { return FULL ? pi : idx; }
  __device__ double ring_at(int row) const { return FULL ? own[row] : ring[row & ring_mask]; }
  // a solved row into the ring, and into the own rows if it is one of them
  __device__ void put_solved(int row, double v) {
    if (FULL) {
      own[row] = v;
    } else {
      ring[row & ring_mask] = v;
      const int t = (row & (kB - 1)) - q * S::R;
      if (t >= 0 && t < S::R) own[(row / kB) * S::R + t] = v;
    }
  }
  // sum over the lanes of a row (lanes of a row differ in the bits above rw)
  template <int rw>
  __device__ static double row_sum(double v) {
#pragma unroll
    for (int o = rw; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
  }

  // GEMV items of round j's s: forward, row i of block j over the columns of
  // blocks <= j - 3; backward, column c of block bt over the rows of blocks
  // >= bt + 3 (both known once round j - 2 has gathered its block).
  __device__ GemvDesc gemv_desc(int j) const {
    GemvDesc d{0, 0, 0, 0, 0};
    if (j < 2 || j >= 2 * nblk || j == nblk) return d;
    if (j < nblk) {
      const int i = j * kB + q * S::R + f_t;
      if (i >= n) return d;
      const int lo = max(0, i - bw), hi = (j - 2) * kB;
      const int c0 = lo + 4 * f_h + f_g, st = 4 * S::H;
      if (c0 >= hi) return d;
      d.cnt = (hi - c0 + st - 1) / st;
      d.off = (int64_t)i * W + (c0 - i + bw);
      d.step = st;
      d.w0 = c0;
      d.wstep = st;
    } else {
      const int bt = 2 * nblk - 1 - j;
      const int c = bt * kB + q * S::R + b_t;
      if (c >= n) return d;
      const int kend = min(n - 1, c + bw);
      const int st = S::KG;
      const int k0 = (bt + 3) * kB + b_kg;
      if (k0 > kend) return d;
      d.cnt = (kend - k0) / st + 1;
      d.off = (int64_t)k0 * W + (c - k0 + bw);
      d.step = (int64_t)st * bw;
      d.w0 = k0;
      d.wstep = st;
    }
    return d;
  }

  // Loads of one GEMV item into registers, stopping at the longest item of
  // the warp (each load instruction costs issue time even when its lanes are off).
  __device__ void gemv_load(const GemvDesc& d, double (&pf)[kPF]) const {
    const int cmax = __reduce_max_sync(kFull, d.cnt);
#pragma unroll
    for (int j = 0; j < kPF; ++j) {
      if (j >= cmax) break;
      pf[j] = j < d.cnt ? __ldg(LB + d.off + j * d.step) : 0.0;
    }
  }

  // Band products of round j's item (values in pf), then the loads of round
  // j + 1 (into pf, cur) so that they overlap the reduction; stores s of the
  // own rows into the ring.  Every FP64 warp instruction costs the same
  // however many lanes are active, so the loop stops at the longest item of
  // the warp; two accumulators halve the dependent chain.
  __device__ void gemv_round(int j, GemvDesc& cur, double (&pf)[kPF]) {
    const int cmax = __reduce_max_sync(kFull, cur.cnt);
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int k = 0; k < kPF; k += 2) {
      if (k >= cmax) break;
      const double x0 = k < cur.cnt ? ring_at(cur.w0 + k * cur.wstep) : 0.0;
      acc0 = fma(pf[k], x0, acc0);
      if (k + 1 >= cmax) break;
      const double x1 = k + 1 < cur.cnt ? ring_at(cur.w0 + (k + 1) * cur.wstep) : 0.0;
      acc1 = fma(pf[k + 1], x1, acc1);
    }
    for (int k = kPF; k < cmax; ++k)
      if (k < cur.cnt)
        acc0 = fma(__ldg(LB + cur.off + k * cur.step), ring_at(cur.w0 + k * cur.wstep), acc0);
    cur = gemv_desc(j + 1);
    gemv_load(cur, pf);
    // a warp without band terms (most rounds of a narrow band) skips its
    // reduction: s = own value exactly, as own - 0 would give
    double* sj = sm.s[j & 3];
    if (j < nblk) {
      double acc = 0.0;
      if (cmax > 0) {
        acc = acc0 + acc1;
        acc += __shfl_xor_sync(kFull, acc, 1);
        acc += __shfl_xor_sync(kFull, acc, 2);
        if (S::H > 1) acc += __shfl_xor_sync(kFull, acc, 4);
        if (S::H > 2) acc += __shfl_xor_sync(kFull, acc, 8);
        if (S::H > 4) acc += __shfl_xor_sync(kFull, acc, 16);
      }
      if (f_g == 0 && f_h == 0) {
        const int row = j * kB + q * S::R + f_t;
        sj[f_t] = row < n ? (cmax > 0 ? own_at(j, f_t) - acc : own_at(j, f_t)) : 0.0;
      }
    } else {
      double acc = 0.0;
      if (cmax > 0) {
        acc = acc0 + acc1;
#pragma unroll
        for (int o = S::TB; o < 32; o <<= 1) acc += __shfl_xor_sync(kFull, acc, o);
      }
      if (b_kg == 0) {
        const int bt = 2 * nblk - 1 - j;
        const int row = bt * kB + q * S::R + b_t;
        sj[b_t] = row < n ? (cmax > 0 ? own_at(bt, b_t) - acc : own_at(bt, b_t)) : 0.0;
      }
    }
  }

  // coupling of round g to the block of round g - 1 for own row t (C1, forward;
  // D1^T, backward; 0 where absent)
  __device__ double c1_val(int g, int t) const {
    const int b = block_of(g), tc = q * S::R + t;
    const int64_t o = (int64_t)b * kBB;
    if (g < nblk) return b >= 1 ? __ldg(C1 + o + tc * kB + x_r) : 0.0;
    return g >= nblk + 1 ? __ldg(D1 + o + tc * kB + x_r) : 0.0;
  }
  __device__ double b_val(int g1, int t) const {
    const int b1 = block_of(g1), tc = q * S::R + t;
    const int64_t o = (int64_t)b1 * kBB;
    return g1 < nblk ? __ldg(BT + o + tc * kB + p_r) : __ldg(B + o + tc * kB + p_r);
  }
  __device__ double c2_val(int g1, int t) const {
    const int b1 = block_of(g1), tc = q * S::R + t;
    const int64_t o = (int64_t)b1 * kBB;
    if (g1 < nblk) return b1 >= 2 ? __ldg(C2 + o + tc * kB + p_r) : 0.0;
    return (g1 != nblk && g1 >= nblk + 2) ? __ldg(D2 + o + tc * kB + p_r) : 0.0;
  }

  __device__ void x_load(int g, double (&pf)[kPF]) const {
    if constexpr (S::PF_X) {
#pragma unroll
      for (int k = 0; k < S::TPX; ++k)
        pf[k] = g < 2 * nblk ? c1_val(g, x_g + S::LPR * k) : 0.0;
    }
  }
  // pre operands of round g1 into registers: B into pf[0, TPP), C2 into
  // pf[TPP, 2 TPP) (each only where it fits)
  __device__ void p_load_b(int g1, double (&pf)[kPF]) const {
    if constexpr (S::PF_B) {
#pragma unroll
      for (int k = 0; k < S::TPP; ++k) pf[k] = g1 < 2 * nblk ? b_val(g1, p_g + S::LPRP * k) : 0.0;
    }
  }
  __device__ void p_load_c2(int g1, double (&pf)[kPF]) const {
    if constexpr (S::PF_C2) {
#pragma unroll
      for (int k = 0; k < S::TPP; ++k)
        pf[S::TPP + k] = g1 < 2 * nblk ? c2_val(g1, p_g + S::LPRP * k) : 0.0;
    }
  }

  // pre of round g1 (lane partial over its own rows): B s - C2 y_{b-2}
  // (forward) or B^T s - D2^T u_{b+2} (backward); the first backward round
  // takes s = y_b (no band part, no couplings).  The B s part needs only s
  // (ready a round before y_{b-2}), so it is taken before the wait for y.
  // B_b is lower triangular (exact zeros above the diagonal): a warp skips
  // the column groups k whose every column lies above its rows (forward, B
  // s) or below them (backward, B^T s) -- products that are exactly zero.
  __device__ double pre_bs(int g1, const double (&pf)[kPF]) const {
    const int b1 = block_of(g1);
    double p0 = 0.0;
    const bool first_bwd = g1 == nblk;
    const double* s1 = sm.s[g1 & 3];
    const int r0 = (warp - S::P0) * S::RWP, r1 = r0 + S::RWP - 1;   // the warp's rows
    const int c0 = q * S::R;                                          // first own column
    // forward: group k is nonzero while c0 + LPRP k <= r1; backward while
    // c0 + LPRP k + LPRP - 1 >= r0
    const int k_end = g1 < nblk ? (r1 - c0 < 0 ? 0 : (r1 - c0) / S::LPRP + 1) : S::TPP;
    const int k_begin = g1 < nblk ? 0 : (r0 - c0 - S::LPRP + 1 <= 0 ? 0
                                          : (r0 - c0 - S::LPRP + 1 + S::LPRP - 1) / S::LPRP);
#pragma unroll
    for (int k = 0; k < S::TPP; ++k) {
      if (k >= k_end) break;
      if (k < k_begin) continue;
      const int t = p_g + S::LPRP * k;
      double bv;
      if constexpr (S::PF_B) bv = pf[k]; else bv = b_val(g1, t);
      p0 = fma(bv, first_bwd ? own_val(b1, t) : s1[t], p0);
    }
    return p0;
  }
  // continues the B s partial p with the C2 term
  __device__ double pre_c2(int g1, const double (&pf)[kPF], double p) const {
    const int b1 = block_of(g1);
    double p1 = p;
    const bool two = g1 < nblk ? b1 >= 2 : g1 >= nblk + 2;
    if (!two) return p1;
    const int bb = block_of(g1 - 2);
#pragma unroll
    for (int k = 0; k < S::TPP; ++k) {
      const int t = p_g + S::LPRP * k;
      double c2;
      if constexpr (S::PF_C2) c2 = pf[S::TPP + k]; else c2 = c2_val(g1, t);
      p1 = fma(-c2, own_val(bb, t), p1);
    }
    return p1;
  }

  // Forward then backward substitution; on return w holds u (all rows).
  __device__ void run(double (&pf)[kPF]) {
    const int G = 2 * nblk;
    if (threadIdx.x == 0) {
      sm.ydone = -1;
      sm.sdone = -1;
      sm.pdone = -1;
      sm.ccount = 0;
    }
    __syncthreads();
    if (is_gemv()) {
      // s of rounds 0 and 1: own right-hand sides (no band part yet)
      const int gt = threadIdx.x - S::GW0 * 32;
      for (int j = 0; j < 2; ++j)
        for (int t = gt; t < S::R; t += S::GW * 32)
          if (j < G && j != nblk) {
            const int row = j * kB + q * S::R + t;
            sm.s[j & 3][t] = row < n ? own_at(j, t) : 0.0;
          }
      if constexpr (CL == 1) {
        // test hook: a wait that runs out of polls sets the error flag; every
        // later wait then returns at once and the lane reports MQS_ST_TIMEOUT.
        // The one-CTA form has no cross-CTA traffic, so nothing is left in
        // flight when the CTA ends.
        if (stall && rounds == 0) wait_count(&sm.sdone, 1 << 30, &sm.err);
      }
      GemvDesc cur = gemv_desc(2);
      gemv_load(cur, pf);
      group_sync(2, S::GW * 32);
      if (gt == 0) st_release(&sm.sdone, 1);
      for (int g = 0; g + 2 < G; ++g) {
        const int j = g + 2;
        wait_count(&sm.ydone, g, &sm.err);
        if (j != nblk) {
          gemv_round(j, cur, pf);
        } else {
          cur = gemv_desc(j + 1);
          gemv_load(cur, pf);
        }
        group_sync(2, S::GW * 32);
        if (gt == 0) st_release(&sm.sdone, j);
      }
    } else if (is_pre()) {
      // pre of every round, one round ahead of the exchange warps, software
      // pipelined: round g1 + 1's B values load while round g1 waits for its
      // C2 operands and its C2 values once round g1's C2 term is formed; its
      // B s part follows the release of round g1, while the exchange warps
      // wait for shares, so that the FP64 pipe is free for their C1 product
      // when the solved block arrives.
      auto bs_of = [&](int g1) -> double {
        if (g1 == nblk)
          wait_count(&sm.ydone, nblk, &sm.err);          // y of the last forward block
        else
          wait_count(&sm.sdone, g1, &sm.err);
        return pre_bs(g1, pf);
      };
      p_load_b(0, pf);
      p_load_c2(0, pf);
      double p0 = bs_of(0);
      for (int g1 = 0; g1 < G; ++g1) {
        if (g1 + 1 < G) p_load_b(g1 + 1, pf);
        if (g1 != nblk) wait_count(&sm.ydone, g1 - 1, &sm.err);   // the block two rounds back
        // the C2 term waits until every exchange warp has its C1 product of
        // the previous round: that product is on the critical path, this one
        // has the share exchange's latency as slack
        if (g1 >= 2 && g1 != nblk) wait_count(&sm.ccount, S::NX * g1, &sm.err);
        const double v = row_sum<S::RWP>(pre_c2(g1, pf, p0));
        if (p_g == 0) sm.pre[g1 & 1][p_r] = v;
        group_sync(3, S::NP * 32);
        if (threadIdx.x == S::P0 * 32) st_release(&sm.pdone, g1);
        if (g1 + 1 < G) {
          p_load_c2(g1 + 1, pf);
          p0 = bs_of(g1 + 1);
        }
      }
    } else if (is_exch()) {
      x_load(0, pf);
      for (int g = 0; g <= G; ++g) {
        // [A] the shares of round g - 1 into the copy (rank order, as a tree)
        if (CL > 1 && g >= 1) {
          const int bp = block_of(g - 1);
          const int64_t r = rounds + g - 1;
          const uint32_t mb = smem_addr(&sm.mbar[r & 1]);
          mbar_wait(mb, (uint32_t)((r >> 1) & 1), &sm.err);
          // round r + 2; after an expired wait the phase may be incomplete and
          // is not armed again
          if (threadIdx.x == 0 && !*reinterpret_cast<volatile int*>(&sm.err))
            mbar_arm(mb, kShareTx<CL>);
          const double* Vb = &sm.V[(g - 1) & 1][0][0];
          constexpr int NV = CL / S::LPR > 0 ? CL / S::LPR : 1;   // shares summed by this lane
          double v[NV];
#pragma unroll
          for (int k = 0; k < NV; ++k) v[k] = Vb[(x_g + S::LPR * k) * kB + x_r];
#pragma unroll
          for (int span = 1; span < NV; span <<= 1)
#pragma unroll
            for (int k = 0; k + span < NV; k += 2 * span) v[k] += v[k + span];
          const double acc = row_sum<S::RW>(v[0]);
          const int row = bp * kB + x_r;
          if (x_g == 0 && row < n) put_solved(row, acc);
        }
        if (g == G) break;
        group_sync(1, S::NX * 32);
        if (threadIdx.x == S::X0 * 32) st_release(&sm.ydone, g);
        const bool fwd = g < nblk;
        const int b = block_of(g);
        // [C] v = pre - C1 y_{b-1} (forward) or pre - D1^T u_{b+1} (backward)
        const bool c1 = fwd ? b >= 1 : g >= nblk + 1;
        const int bp = block_of(g - 1);
        wait_count(&sm.pdone, g, &sm.err);
        double v0 = x_g == 0 ? sm.pre[g & 1][x_r] : 0.0, v1 = 0.0;
        if (c1) {
#pragma unroll
          for (int k = 0; k < S::TPX; ++k) {
            const int t = x_g + S::LPR * k;
            double c;
            if constexpr (S::PF_X) c = pf[k]; else c = c1_val(g, t);
            if (k & 1)
              v1 = fma(-c, own_val(bp, t), v1);
            else
              v0 = fma(-c, own_val(bp, t), v0);
          }
        }
        const double v = row_sum<S::RW>(v0 + v1);
        // next round's C1 values; with 4 and 8 CTAs (3 and 7 remote stores
        // per lane) before the shares, so that these loads do not queue
        // behind the stores -- measured faster there, slower with 2 CTAs
        if constexpr (CL >= 4) x_load(g + 1, pf);
        __syncwarp();
        if ((threadIdx.x & 31) == 0) atomicAdd(&sm.ccount, 1);
        if constexpr (CL == 1) {
          const int row = b * kB + x_r;
          if (x_g == 0 && row < n) put_solved(row, v);
        } else {
          const uint32_t la = smem_addr(&sm.V[g & 1][q][x_r]);
          const uint32_t lm = smem_addr(&sm.mbar[g & 1]);
          // after an expired wait this CTA's values are invalid: it stops
          // sending, so the other CTAs' waits run out too and the lane leaves
          // at the next step boundary
          const bool failed = *reinterpret_cast<volatile int*>(&sm.err) != 0;
          for (int p = x_g; p < CL; p += S::LPR) {
            if (p == q)
              sm.V[g & 1][q][x_r] = v;   // own share: ordered by the group barrier of the next round
            else if (!failed)
              st_async(map_rank(la, p), v, map_rank(lm, p));
          }
        }
        if constexpr (CL < 4) x_load(g + 1, pf);
      }
    }
    __syncthreads();
    rounds += G;
  }
};

// ---------------------------------------------------------------- stepping
// Own nodes of rank q: band rows pi with (pi mod 64) in [q*R, q*R + R), R = 64/CL.
template <int CL>
struct Own {
  int n, q;
  __device__ int count() const { return ((n + kB - 1) / kB) * Split<CL>::R; }
  __device__ int row(int idx) const {
    constexpr int R = Split<CL>::R;
    return (idx / R) * kB + q * R + idx % R;
  }
};

// Error flag cleared; mbarriers of the share exchange (CL > 1) initialised
// once, each armed one round ahead (rounds 0 and 1 here, round r + 2 when
// round r's shares are consumed).
template <int CL>
__device__ void cluster_setup(CSmem<CL>& sm) {
  if (threadIdx.x == 0) sm.err = 0;
  if constexpr (CL == 1) {
    __syncthreads();
  } else {
    if (threadIdx.x == 0) {
      for (int x = 0; x < 2; ++x) {
        const uint32_t mb = smem_addr(&sm.mbar[x]);
        mbar_init(mb);
        mbar_arm(mb, kShareTx<CL>);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync_all();
  }
}

// No CTA leaves while shares may still be sent to it; a timed-out wait (of
// any cluster size) is reported on the lane's status.
template <int CL>
__device__ void cluster_finish(CSmem<CL>& sm, const DirectLane& D) {
  if constexpr (CL > 1) {
    cluster_sync_all();
  } else {
    __syncthreads();
  }
  if (threadIdx.x == 0 && sm.err && D.status_out) atomicOr(D.status_out, MQS_ST_TIMEOUT);
}

// Flags of a step boundary, identical on every CTA of the cluster: each CTA
// publishes its error flag (bit 0) and rank 0 the cancellation state (bit 1)
// into slot `slot` before the barrier; after it every CTA ors the slots of all
// ranks.  A slot is written again two boundaries later, after a barrier that
// every CTA passes only once it has read the slot.
// System-scope load of a word the host writes (host-mapped memory).
__device__ __forceinline__ int32_t load_sys(const volatile int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int CL>
__device__ int boundary_flags(CSmem<CL>& sm, const DirectConst& kc, unsigned q, int slot) {
  if (threadIdx.x == 0) {
    int f = *reinterpret_cast<volatile int*>(&sm.err) ? 1 : 0;
    if (q == 0 && kc.stop && load_sys(kc.stop) < kc.iter) f |= 2;
    sm.flag_pub[slot] = f;
  }
  int f = 0;
  if constexpr (CL == 1) {
    __syncthreads();
    f = *reinterpret_cast<volatile int*>(&sm.flag_pub[slot]);
  } else {
    cluster_sync_all();
    cg::cluster_group cl = cg::this_cluster();
    for (int p = 0; p < CL; ++p) f |= *cl.map_shared_rank(&sm.flag_pub[slot], p);
  }
  return f;
}

// Advance one lane by n_steps steps.  a_init: initial state (all nodes
// readable) or nullptr for zero; on return the final state is in D.a0 (own
// nodes).  Returns this thread's share of the raw QoI sum when want_qoi.
// `left` receives the step-boundary flags that ended the run early (1: a wait
// ran out, 2: the launch was cancelled; 0: all steps ran), the same on every
// CTA of the cluster.
template <int CL, bool FULL>
__device__ double cluster_integrate(const DirectConst& kc, const DirectLane& D,
                                    const double* a_init, int n_steps, int64_t k0, unsigned q,
                                    Subst<CL, FULL>& sub, double* own_w, bool want_qoi, int& left) {
  left = 0;
  if (kc.stop) {   // a launch queued behind the iteration that met the stopping rule
    left = boundary_flags<CL>(sub.sm, kc, q, 1);
    if (left) return 0.0;
  }
  const int n = kc.n;
  const Own<CL> own{n, (int)q};
  const int n_own = own.count();
  double* a0 = D.a0;
  double* a1 = D.a1;
  double* y = D.y;
  const double* Mv = kc.M + D.vcol;
  const double* Kv = kc.K ? kc.K + D.vcol : nullptr;
  for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
    const int pi = own.row(idx);
    if (pi >= n) continue;
    const int i = __ldg(kc.perm + pi);
    if (a_init) {
      y[i] = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a_init);
      if (a_init != a0) a0[i] = a_init[i];
    } else {
      a0[i] = 0.0;
      y[i] = 0.0;
    }
  }
  double pf[kPF];
  double qacc = 0.0;
  const double dt = D.dt, inv_dt = 1.0 / D.dt;
  for (int step = 0; step < n_steps; ++step) {
    const double t = D.t0 + (double)(k0 + step + 1) * dt;
    double gph[kMaxPhases];
#pragma unroll
    for (int ph = 0; ph < kMaxPhases; ++ph) {
      gph[ph] = 0.0;
      if (ph < kc.n_phases) {
        const double arg = kc.omega * t - (2.0 * kPi * ph) / kc.n_phases + D.phase[ph];
        gph[ph] = D.amp[ph] * sin(arg);
      }
    }
    for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
      const int pi = own.row(idx);
      if (pi >= n) continue;
      const int i = __ldg(kc.perm + pi);
      double f = 0.0;
#pragma unroll
      for (int ph = 0; ph < kMaxPhases; ++ph)
        if (ph < kc.n_phases) f = fma(gph[ph], __ldg(kc.F + (int64_t)ph * n + i), f);
      own_w[sub.own_index(idx, pi)] = fma(y[i], inv_dt, f) * __ldg(D.invd + pi);   // D^-1 b
    }
    __syncthreads();
    sub.run(pf);
    for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
      const int pi = own.row(idx);
      if (pi >= n) continue;
      const int i = __ldg(kc.perm + pi);
      a1[i] = own_w[sub.own_index(idx, pi)] * __ldg(D.invd + pi);   // x = D^-1 u
    }
    // a1 complete for y = M a1; the whole cluster leaves here together after
    // an expired wait or a cancellation
    left = boundary_flags<CL>(sub.sm, kc, q, step & 1);
    if (left) return qacc;
    for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
      const int pi = own.row(idx);
      if (pi >= n) continue;
      const int i = __ldg(kc.perm + pi);
      const double yn = csr_row(kc.rowptr, kc.colidx, i, Mv, kc.vs, a1);
      if (want_qoi) {
        if (kc.qoi_kind == MQS_QOI_JOULE)
          qacc = fma(a1[i] - a0[i], yn - y[i], qacc);
        else
          qacc = fma(a1[i], csr_row(kc.rowptr, kc.colidx, i, Kv, kc.vs, a1), qacc);
      }
      y[i] = yn;
    }
    double* tmp = a0;
    a0 = a1;
    a1 = tmp;
  }
  if (n_steps & 1) {
    for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
      const int pi = own.row(idx);
      if (pi >= n) continue;
      const int i = __ldg(kc.perm + pi);
      a1[i] = a0[i];
    }
  }
  __syncthreads();
  return qacc;
}

template <int CL, bool FULL>
__global__ void __launch_bounds__(kNT, 1) k_cluster_propagate(const DirectLane* __restrict__ lanes,
                                                            DirectConst kc) {
  __shared__ CSmem<CL> sm;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  double* own = reinterpret_cast<double*>(dyn_smem);
  const int ring_rows = cluster_ring_rows(kc.bw);
  double* ring = FULL ? own : own + own_rows<CL>(kc.n);
  const unsigned q = CL > 1 ? cluster_rank() : 0u;
  const DirectLane D = lanes[blockIdx.x / CL];
  cluster_setup<CL>(sm);
  Subst<CL, FULL> sub(D, own, ring, ring_rows, sm, kc.n, kc.bw, (int)q);
  sub.stall = kc.stall_test != 0;
  const double* init = D.init_from_a0 ? (D.a_init ? D.a_init : D.a0) : nullptr;
  int left = 0;
  const double part = cluster_integrate<CL, FULL>(kc, D, init, D.n_steps, D.k0, q, sub, own,
                                                  true, left);
  const double s = cluster_sum<CL>(cta_sum(part, sm.red), sm, 0, q);
  if (threadIdx.x == 0 && q == 0)
    D.qoi_out[0] = (kc.qoi_kind == MQS_QOI_JOULE ? s / D.dt : 0.5 * s) * D.qoi_scale;
  cluster_finish<CL>(sm, D);
}

// Parareal coarse sweep (Eq. 12), one cluster per sample; slice states
// lane-major U/E/G[(sample*M + s) * n + i].
template <int CL, bool FULL>
__global__ void __launch_bounds__(kNT, 1) k_cluster_chain(const DirectLane* __restrict__ lanes,
                                                        DirectConst kc, DirectChain ch) {
  __shared__ CSmem<CL> sm;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  double* own_w = reinterpret_cast<double*>(dyn_smem);
  const int ring_rows = cluster_ring_rows(kc.bw);
  double* ring = FULL ? own_w : own_w + own_rows<CL>(kc.n);
  const unsigned q = CL > 1 ? cluster_rank() : 0u;
  const DirectLane D = lanes[blockIdx.x / CL];
  const int n = kc.n;
  const Own<CL> own{n, (int)q};
  const int n_own = own.count();
  const int sample = D.sample;
  cluster_setup<CL>(sm);
  Subst<CL, FULL> sub(D, own_w, ring, ring_rows, sm, n, kc.bw, (int)q);
  sub.stall = kc.stall_test != 0;
  const int s_stop = min(ch.s_end, ch.M - 1);
  for (int s = ch.s_begin; s < s_stop; ++s) {
    const int64_t base = ((int64_t)sample * ch.M + s) * n;
    const double* U0 = s == ch.s_first ? ch.U_prev : ch.U_cur;
    int left = 0;
    cluster_integrate<CL, FULL>(kc, D, U0 + base, ch.steps_per_slice,
                                (int64_t)s * ch.steps_per_slice, q, sub, own_w, false, left);
    if (left) break;   // every CTA of the cluster leaves at the same slice
    double j2 = 0.0, u2 = 0.0;
    for (int idx = threadIdx.x; idx < n_own; idx += kNT) {
      const int pi = own.row(idx);
      if (pi >= n) continue;
      const int i = __ldg(kc.perm + pi);
      const double gn = D.a0[i];
      const double un = ch.first_sweep ? gn : ch.E[base + i] + (gn - ch.G[base + i]);
      const double du = un - ch.U_prev[base + n + i];
      j2 = fma(du, du, j2);
      u2 = fma(un, un, u2);
      ch.U_cur[base + n + i] = un;
      ch.G[base + i] = gn;
    }
    j2 = cluster_sum<CL>(cta_sum(j2, sm.red), sm, 0, q);
    u2 = cluster_sum<CL>(cta_sum(u2, sm.red), sm, 1, q);   // also publishes U[s + 1]
    if (threadIdx.x == 0 && q == 0) {
      ch.jump2[(int64_t)sample * ch.M + s + 1] = j2;
      ch.norm2[(int64_t)sample * ch.M + s + 1] = u2;
    }
    __syncthreads();
  }
  cluster_finish<CL>(sm, D);
}

// ---------------------------------------------------------------- block preparation
// One CTA per (64-row block b, factor): the inverse B_b of the unit lower
// diagonal block of L~ (identity rows past n) by forward substitution, one
// thread per column, then the couplings as dense products: C1_b = B_b
// L~_{b,b-1}, C2_b = B_b L~_{b,b-2}; D1_b^T = L~_{b+1,b} B_b, D2_b^T =
// L~_{b+2,b} B_b (zero where the block is absent).  Everything the forward
// sweep reads (B_b, C1_b, C2_b) is stored column-major [t][r] and what the
// backward sweep reads (B_b^T, D1_b^T, D2_b^T) as [t][r] of the transpose,
// i.e. B_b row-major [r][t]: a lane of the stepping kernels takes one row r,
// consecutive lanes consecutive rows, so every load of a warp is coalesced.
constexpr int kPrepThreads = 256;

__global__ void __launch_bounds__(kPrepThreads) k_block_prep(const double* __restrict__ LBall, int n,
                                                            int bw, int64_t fstride, int nblk,
                                                            double* __restrict__ B_all,
                                                            double* __restrict__ BT_all,
                                                            double* __restrict__ C1_all,
                                                            double* __restrict__ C2_all,
                                                            double* __restrict__ D1_all,
                                                            double* __restrict__ D2_all) {
  extern __shared__ __align__(16) unsigned char prep_smem[];
  double (*O)[kB + 1] = reinterpret_cast<double (*)[kB + 1]>(prep_smem);
  double (*Bs)[kB + 1] = reinterpret_cast<double (*)[kB + 1]>(prep_smem + sizeof(double) * kB * (kB + 1));
  const int b = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
  const double* LB = LBall + f * fstride;
  const int64_t bo = ((int64_t)f * nblk + b) * kB * kB;
  const int W = bw + 1;
  // L~(64 bi + m, 64 bj + cc), zero outside the matrix, above the diagonal and outside the band
  auto blk = [&](int bi, int bj, int m, int cc) -> double {
    if (bi < 0 || bi >= nblk || bj < 0) return 0.0;
    const int i = bi * kB + m, col = bj * kB + cc;
    if (i >= n || col > i || i - col > bw) return 0.0;
    return LB[(int64_t)i * W + (col - i + bw)];
  };
  for (int e = tid; e < kB * kB; e += kPrepThreads) {
    const int r = e / kB, c = e % kB;
    O[r][c] = b * kB + r < n ? blk(b, b, r, c) : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  if (tid < kB) {   // column c of the inverse
    const int c = tid;
    for (int r = 0; r < kB; ++r) {
      double x = r == c ? 1.0 : 0.0;
      for (int j = c; j < r; ++j) x = fma(-O[r][j], Bs[j][c], x);
      Bs[r][c] = x;
    }
  }
  __syncthreads();
  for (int e = tid; e < kB * kB; e += kPrepThreads) {
    B_all[bo + e] = Bs[e / kB][e % kB];
    BT_all[bo + e] = Bs[e % kB][e / kB];
  }
  double* outs[4] = {C1_all, C2_all, D1_all, D2_all};
  for (int which = 0; which < 4; ++which) {
    __syncthreads();
    for (int e = tid; e < kB * kB; e += kPrepThreads) {
      const int r = e / kB, c = e % kB;
      O[r][c] = which == 0 ? blk(b, b - 1, r, c)
              : which == 1 ? blk(b, b - 2, r, c)
              : which == 2 ? blk(b + 1, b, r, c)
                           : blk(b + 2, b, r, c);
    }
    __syncthreads();
    for (int e = tid; e < kB * kB; e += kPrepThreads) {
      // C1, C2 column-major: element (r, c) at [c][r]; D1^T, D2^T as computed
      const int r = which < 2 ? e % kB : e / kB, c = which < 2 ? e / kB : e % kB;
      double a0 = 0.0, a1 = 0.0;
      if (which < 2) {
#pragma unroll 8
        for (int m = 0; m < kB; m += 2) {
          a0 = fma(Bs[r][m], O[m][c], a0);
          a1 = fma(Bs[r][m + 1], O[m + 1][c], a1);
        }
      } else {
#pragma unroll 8
        for (int m = 0; m < kB; m += 2) {
          a0 = fma(O[r][m], Bs[m][c], a0);
          a1 = fma(O[r][m + 1], Bs[m + 1][c], a1);
        }
      }
      outs[which][bo + e] = a0 + a1;
    }
  }
}

// ---------------------------------------------------------------- band Cholesky on a cluster
// Right-looking band Cholesky of one factor on a cluster of NC CTAs (the same
// result and layout as the one-CTA k_band_chol: L in place, L(j, j) on the
// diagonal, invd = 1 / L(j, j); the products of the trailing updates summed in
// a separate accumulator S and subtracted once, as there).  Row i belongs to
// CTA i mod NC, which keeps it (and its S row) in a shared-memory ring from
// the column where it enters the band window until it is final, then writes
// it back once.  Per column j: every CTA
// scales its rows' entry of column j and sends it to every CTA's column
// buffer; the owner of row j + 1 forms that row's pivot and sends its
// reciprocal; all sends are asynchronous DSMEM stores counted on the
// receiver's mbarrier.  Then every CTA applies the rank-1 update to its rows.
__device__ __forceinline__ int count_mod(int a, int b, int r, int nc) {   // #{i in [a, b]: i % nc == r}
  if (b < a) return 0;
  const int first = a + ((r - a) % nc + nc) % nc;
  return first > b ? 0 : (b - first) / nc + 1;
}

template <int NC>
struct CholRing {
  static int slots(int bw) { return (bw + 1 + NC - 1) / NC + 2; }
  static size_t bytes(int bw) {   // rows and S rows of the ring, two column buffers
    return sizeof(double) * (2 * (size_t)slots(bw) * (bw + 1) + 2 * (size_t)std::max(bw, 1));
  }
};

template <int NC>
__global__ void __launch_bounds__(kNT, 1) k_band_chol_cl(double* __restrict__ LBall,
                                                       double* __restrict__ invd_all, int n, int bw,
                                                       int64_t fstride, int32_t* __restrict__ bad) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  const int W = bw + 1;
  const int RING = (bw + 1 + NC - 1) / NC + 2;
  double* ring = reinterpret_cast<double*>(chol_smem);   // [RING][W]: own rows of the window
  double* sring = ring + (size_t)RING * W;                // [RING][W]: their accumulated products
  double* col = sring + (size_t)RING * W;                 // [2][bw]: column j of L below the diagonal
  __shared__ double piv[2];                               // 1 / L(j, j) by column parity
  __shared__ double l00;
  __shared__ unsigned long long mb[2];
  __shared__ int err;
  const int rho = (int)cluster_rank();
  const int f = blockIdx.x / NC;
  double* LB = LBall + f * fstride;
  double* invd = invd_all + (int64_t)f * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto row_of = [&](int i) -> double* { return ring + (size_t)((i / NC) % RING) * W; };
  auto srow_of = [&](int i) -> double* { return sring + (size_t)((i / NC) % RING) * W; };
  auto load_row = [&](int i) {          // all threads of the CTA
    const double* src = LB + (int64_t)i * W;
    double* dst = row_of(i);
    double* sd = srow_of(i);
    for (int d = threadIdx.x; d < W; d += kNT) {
      dst[d] = src[d];
      sd[d] = 0.0;
    }
  };
  auto store_row = [&](int i) {
    const double* src = row_of(i);
    double* dst = LB + (int64_t)i * W;
    for (int d = threadIdx.x; d < W; d += kNT) dst[d] = src[d];
  };
  // bytes this CTA receives for column j: the other CTAs' rows and the next pivot
  auto tx_of = [&](int j) -> uint32_t {
    if (j >= n) return 0u;
    const int total = min(bw, n - 1 - j);
    const int own = count_mod(j + 1, j + total, rho, NC);
    const int pv = (j + 1 < n && (j + 1) % NC != rho) ? 1 : 0;
    return (uint32_t)((total - own + pv) * sizeof(double));
  };
  for (int i = rho; i < min(n, bw + 1); i += NC) load_row(i);   // rows in the window of column 0
  if (threadIdx.x == 0) {
    err = 0;
    for (int x = 0; x < 2; ++x) {
      mbar_init(smem_addr(&mb[x]));
      mbar_arm(smem_addr(&mb[x]), tx_of(x));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    double d = LB[bw];   // every CTA forms the first pivot from A(0, 0)
    if (!(d > 0.0)) {
      if (rho == 0) bad[f] = 1;
      d = 1.0;
    }
    l00 = sqrt(d);
    piv[0] = 1.0 / l00;
  }
  cluster_sync_all();   // A(0, 0) read everywhere before CTA 0 writes row 0 back
  if (rho == 0) {
    if (threadIdx.x == 0) {
      row_of(0)[bw] = l00;
      invd[0] = piv[0];
    }
    __syncthreads();
    store_row(0);
  }
  for (int j = 0; j < n; ++j) {
    const int par = j & 1;
    const int total = min(bw, n - 1 - j);
    const double inv = piv[par];
    double* cj = col + par * bw;
    // own rows of column j: i = first + NC k, i in (j, j + total]
    const int first = j + 1 + ((rho - (j + 1)) % NC + NC) % NC;
    const int n_own = first > j + total ? 0 : (j + total - first) / NC + 1;
    if (threadIdx.x < n_own) {
      const int i = first + NC * threadIdx.x;
      double* row = row_of(i);
      double* srw = srow_of(i);
      const double l = (row[j - i + bw] - srw[j - i + bw]) * inv;
      row[j - i + bw] = l;
      const uint32_t la = smem_addr(cj + (i - j - 1));
      const uint32_t lm = smem_addr(&mb[par]);
      for (int p = 0; p < NC; ++p) {
        if (p == rho)
          cj[i - j - 1] = l;
        else
          st_async(map_rank(la, p), l, map_rank(lm, p));
      }
      if (i == j + 1) {   // this CTA owns row j + 1: its pivot
        // the last product of the diagonal, then A - S, as in k_band_chol
        double d = row[bw] - fma(l, l, srw[bw]);
        if (!(d > 0.0)) {
          bad[f] = 1;
          d = 1.0;
        }
        const double L = sqrt(d);
        const double r = 1.0 / L;
        row[bw] = L;
        invd[j + 1] = r;
        const uint32_t pa = smem_addr(&piv[par ^ 1]);
        for (int p = 0; p < NC; ++p) {
          if (p == rho)
            piv[par ^ 1] = r;
          else
            st_async(map_rank(pa, p), r, map_rank(lm, p));
        }
      }
    }
    mbar_wait(smem_addr(&mb[par]), (uint32_t)((j >> 1) & 1), &err);
    __syncthreads();
    if (threadIdx.x == 0 && !err) mbar_arm(smem_addr(&mb[par]), tx_of(j + 2));   // column j + 2
    // rank-1 update of the own rows (j + 1, j + total], entries j + 1 .. i
    for (int k = warp; k < n_own; k += kNW) {
      const int i = first + NC * k;
      if (i == j + 1) continue;
      const double li = cj[i - j - 1];
      double* srw = srow_of(i) + bw - i;                // srw[c] = S(i, c)
      for (int c = j + 1 + lane; c <= i; c += 32) srw[c] = fma(li, cj[c - j - 1], srw[c]);
    }
    // row j + 1 is final: write it back; row j + 1 + bw enters the window at column j + 1
    if (j + 1 < n && (j + 1) % NC == rho) store_row(j + 1);
    if (j + 1 + bw < n && (j + 1 + bw) % NC == rho) load_row(j + 1 + bw);
    __syncthreads();
  }
  cluster_sync_all();
  if (threadIdx.x == 0 && err) bad[f] = 1;
}

// ---------------------------------------------------------------- launch helpers
template <int CL, bool FULL>
const void* propagate_fn() { return reinterpret_cast<const void*>(&k_cluster_propagate<CL, FULL>); }
template <int CL, bool FULL>
const void* chain_fn() { return reinterpret_cast<const void*>(&k_cluster_chain<CL, FULL>); }

template <int CL>
size_t cluster_smem_t(int n, int bw) {
  return (size_t)(own_rows<CL>(n) + cluster_ring_rows(bw)) * sizeof(double);
}
// Shared memory of the own-rows + ring layout.
size_t cluster_ring_smem(int n, int bw, int CL) {
  switch (CL) {
    case 1: return cluster_smem_t<1>(n, bw);
    case 2: return cluster_smem_t<2>(n, bw);
    case 4: return cluster_smem_t<4>(n, bw);
    default: return cluster_smem_t<8>(n, bw);
  }
}
size_t fixed_smem(int CL) {
  switch (CL) {
    case 1: return sizeof(CSmem<1>);
    case 2: return sizeof(CSmem<2>);
    case 4: return sizeof(CSmem<4>);
    default: return sizeof(CSmem<8>);
  }
}
// The full work vector fits next to the static shared memory; env
// MQS_CLUSTER_RING=1 takes the own-rows + ring layout anyway (for tests: both
// layouts give bitwise the same results).
bool cluster_full(int n, int CL) {
  const char* v = getenv("MQS_CLUSTER_RING");
  const bool force_ring = v && *v && atoi(v) != 0;
  return !force_ring && (size_t)n * sizeof(double) + fixed_smem(CL) + 1024 <= 227 * 1024;
}
size_t cluster_smem(int n, int bw, int CL) {
  return cluster_full(n, CL) ? (size_t)n * sizeof(double) : cluster_ring_smem(n, bw, CL);
}

template <int CL, bool FULL>
int set_attrs(size_t smem) {
  MQS_CUDA_TRY(cudaFuncSetAttribute(propagate_fn<CL, FULL>(),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MQS_CUDA_TRY(cudaFuncSetAttribute(chain_fn<CL, FULL>(),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return MQS_OK;
}

template <int CL, bool FULL, class... Args>
int launch_cl(const void* fn, int n_lanes, size_t smem, cudaStream_t st, Args... args) {
  MQS_TRY((set_attrs<CL, FULL>(smem)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_lanes * CL));
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* argv[] = {(void*)&args...};
  MQS_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, argv));
  count_launch();
  return MQS_OK;
}

template <int CL, bool FULL>
int max_active_t(size_t smem) {
  if (set_attrs<CL, FULL>(smem) != MQS_OK) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)CL);
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, propagate_fn<CL, FULL>(), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

}  // namespace

// The work vector (full copy, or own rows and the ring) fits next to the static
// shared memory (227 KB per CTA).
bool cluster_fits(int n, int bw, int CL) {
  return cluster_smem(n, bw, CL) + fixed_smem(CL) + 1024 <= 227 * 1024;
}

int cluster_max_active(int CL, int n, int bw) {
  static std::mutex mu;
  static int cache[4][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
  static int64_t cache_n[4] = {-1, -1, -1, -1};
  const int slot = CL == 1 ? 0 : CL == 2 ? 1 : CL == 4 ? 2 : CL == 8 ? 3 : -1;
  if (slot < 0 || !cluster_fits(n, bw, CL)) return 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const bool full = cluster_full(n, CL);
  const int64_t key = ((int64_t)n * 65536 + bw) * 2 + (full ? 1 : 0);
  std::lock_guard<std::mutex> lk(mu);
  if (cache_n[slot] == key && cache[slot][0] == dev) return cache[slot][1];
  const size_t smem = cluster_smem(n, bw, CL);
  int r = 0;
  switch (CL) {
    case 1: r = full ? max_active_t<1, true>(smem) : max_active_t<1, false>(smem); break;
    case 2: r = full ? max_active_t<2, true>(smem) : max_active_t<2, false>(smem); break;
    case 4: r = full ? max_active_t<4, true>(smem) : max_active_t<4, false>(smem); break;
    case 8: r = full ? max_active_t<8, true>(smem) : max_active_t<8, false>(smem); break;
  }
  cache_n[slot] = key;
  cache[slot][0] = dev;
  cache[slot][1] = r;
  return r;
}

int cluster_block_rows() { return kB; }

// Band Cholesky of n_fac factors, one cluster of 8 CTAs each (see
// k_band_chol_cl); MQS_ENOTSUP-style refusal is left to the caller, which
// uses the one-CTA kernel when the factors fill the GPU.
int band_chol_cluster(double* LB, double* invd, int n, int bw, int64_t fstride, int n_fac,
                      int32_t* bad, cudaStream_t st) {
  constexpr int NC = 8;
  if (n_fac <= 0) return MQS_OK;
  const size_t smem = CholRing<NC>::bytes(bw);
  MQS_CUDA_TRY(cudaFuncSetAttribute(k_band_chol_cl<NC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_fac * NC));
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  MQS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_chol_cl<NC>, LB, invd, n, bw, fstride, bad));
  count_launch();
  return MQS_OK;
}
int band_chol_cluster_size() { return 8; }
// The cluster kernel keeps the window's rows and their accumulated products in
// shared memory: bandwidths up to ~300 on 8 CTAs.
bool band_chol_cluster_fits(int bw) { return CholRing<8>::bytes(bw) <= 200 * 1024; }

int block_prep(const MeshDev& m, int n_fac, const double* LB, double* B, double* BT, double* C1,
               double* C2, double* D1, double* D2, cudaStream_t st) {
  const int nblk = (m.n_free + kB - 1) / kB;
  const int64_t fstride = (int64_t)m.n_free * (m.bw + 1);
  if (n_fac <= 0) return MQS_OK;
  const size_t smem = 2 * sizeof(double) * kB * (kB + 1);
  MQS_CUDA_TRY(cudaFuncSetAttribute(k_block_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  k_block_prep<<<dim3((unsigned)nblk, (unsigned)n_fac), kPrepThreads, smem, st>>>(
      LB, m.n_free, m.bw, fstride, nblk, B, BT, C1, C2, D1, D2);
  MQS_CUDA_TRY(cudaGetLastError());
  count_launch();
  return MQS_OK;
}

namespace {
template <int CL, class... Args>
int launch_layout(bool chain, bool full, int n_lanes, size_t smem, cudaStream_t st,
                  Args... args) {
  if (full)
    return launch_cl<CL, true>(chain ? chain_fn<CL, true>() : propagate_fn<CL, true>(), n_lanes,
                               smem, st, args...);
  return launch_cl<CL, false>(chain ? chain_fn<CL, false>() : propagate_fn<CL, false>(), n_lanes,
                              smem, st, args...);
}
}  // namespace

int launch_cluster(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc, cudaStream_t st) {
  if (n_lanes <= 0) return MQS_OK;
  const size_t smem = cluster_smem(kc.n, kc.bw, kc.cluster);
  const bool full = cluster_full(kc.n, kc.cluster);
  switch (kc.cluster) {
    case 1: return launch_layout<1>(false, full, n_lanes, smem, st, d_lanes, kc);
    case 2: return launch_layout<2>(false, full, n_lanes, smem, st, d_lanes, kc);
    case 4: return launch_layout<4>(false, full, n_lanes, smem, st, d_lanes, kc);
    case 8: return launch_layout<8>(false, full, n_lanes, smem, st, d_lanes, kc);
  }
  set_error("unsupported cluster size %d", kc.cluster);
  return MQS_EINVAL;
}

int launch_cluster_chain(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                         const DirectChain& ch, cudaStream_t st) {
  if (n_lanes <= 0) return MQS_OK;
  const size_t smem = cluster_smem(kc.n, kc.bw, kc.cluster);
  const bool full = cluster_full(kc.n, kc.cluster);
  switch (kc.cluster) {
    case 1: return launch_layout<1>(true, full, n_lanes, smem, st, d_lanes, kc, ch);
    case 2: return launch_layout<2>(true, full, n_lanes, smem, st, d_lanes, kc, ch);
    case 4: return launch_layout<4>(true, full, n_lanes, smem, st, d_lanes, kc, ch);
    case 8: return launch_layout<8>(true, full, n_lanes, smem, st, d_lanes, kc, ch);
  }
  set_error("unsupported cluster size %d", kc.cluster);
  return MQS_EINVAL;
}

}  // namespace mqs
