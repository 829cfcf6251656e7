// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "mqs.h"

namespace mqs {

constexpr int kMaxRegions = 16;
constexpr int kMaxPhases = 4;
constexpr int kMaxRowNnz = 32;

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define MQS_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::mqs::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                       __FILE__, __LINE__);                                        \
      return MQS_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define MQS_TRY(expr)             \
  do {                            \
    int s_ = (expr);              \
    if (s_ != MQS_OK) return s_;  \
  } while (0)

// ---------------------------------------------------------------- device buffer
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // (Re)allocate to at least `n` bytes; contents undefined.
  int ensure(size_t n) {
    if (n <= bytes && p) return MQS_OK;
    release();
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMalloc(%zu bytes) failed: %s", n, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? MQS_ENOMEM : MQS_ECUDA;
    }
    bytes = n;
    return MQS_OK;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------- mesh
struct MeshDev {
  int32_t n_nodes = 0, n_tri = 0, n_regions = 0, n_phases = 0;
  int32_t n_free = 0;
  int64_t nnz = 0;
  int32_t max_row_nnz = 0;
  DevBuf rowptr, colidx, diag;   // CSR pattern over free unknowns (int32)
  DevBuf Mr, Kr;                 // [R][nnz] region reference matrices (double)
  DevBuf F;                      // [P][n_free] per-phase load vectors (double)
  std::vector<int32_t> free_node;
  int live_batches = 0;
  // banded direct solver: reverse Cuthill-McKee ordering of the free unknowns
  int32_t bw = -1;               // lower bandwidth in the new ordering (-1: not built)
  DevBuf perm, iperm;            // perm[new] = old, iperm[old] = new (int32)
  DevBuf band_idx;               // [nnz] position of a lower-band entry in [n][bw+1], -1 above
};

// Reverse Cuthill-McKee ordering of a symmetric CSR pattern (host); boundary
// ([n], or empty) marks the nodes next to the Dirichlet boundary, whose pieces
// give a second candidate start set (the narrower band is kept).
void rcm_order(int n, const std::vector<int32_t>& rowptr, const std::vector<int32_t>& colidx,
               const std::vector<char>& boundary, std::vector<int32_t>& perm,
               int32_t& bandwidth);

// ---------------------------------------------------------------- solve lanes
// One tile = L consecutive lanes that share a step size and a step count and
// are advanced together by one cluster ("team") of CTAs.
struct TileDesc {
  // matrix values of lane l of this tile: element k at vals[k * vs + l * ls]
  const double* A;
  const double* M;
  const double* K;       // stiffness values (energy QoI only, else nullptr)
  const float* A32;      // FP32 copy of A (mixed precision only)
  const double* Dinv;    // inverse diagonal of A: row i at Dinv[i * ds + l * ls]
  int64_t vs, ds;
  int32_t ls;            // 1: per-lane values, 0: one value column for the tile
  int32_t lane0;         // first lane of the tile in the batch-wide lane arrays
  // lane vectors: element (i, l) at v[i * xs + l]; pointers include the tile offset
  double *a0, *a1, *y, *r, *p, *q, *z, *b;
  float *p32, *q32;
  int64_t xs;
  double dt, t0;
  int32_t n_steps;
  int32_t n_active;      // lanes [0, n_active) of the tile are real
  int32_t init_from_a0;  // 1: a0 holds the initial state, 0: start from zero
  int32_t pad_;
};

// per-lane data in batch-wide arrays (index = lane0 + l)
struct LaneArrays {
  const double* src_amp;   // [lanes][kMaxPhases]  J0 * amp_p
  const double* src_phi;   // [lanes][kMaxPhases]  phase_p
  const int32_t* k0;       // [lanes] global index of the first step
  double* qoi_raw;         // [lanes] raw QoI sum
  int32_t* status;         // [lanes] MQS_ST_* bits (or-ed)
  double* iters;           // [lanes] total PCG iterations (accumulated)
};

struct TeamConst {
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* F;         // [P][n]
  int32_t n;
  int32_t n_phases;
  int32_t qoi_kind;
  int32_t max_it;
  int32_t replace_every;   // mixed precision: FP64 residual replacement period
  int32_t pad_;
  double tol2;             // cg_tol^2
  double omega;            // 2 pi f
  LaneArrays lanes;
};

// Parareal coarse chain: lane l of the chain is sample (chain_lane0 + l);
// slice state arrays are in the fine-batch lane layout (lane = sample * M + s).
struct ChainDesc {
  double *U, *E, *G;       // [n][xs_par] slice starts, fine ends, previous coarse ends
  int64_t xs_par;
  int32_t M;               // slices per sample
  int32_t s_begin;         // first slice whose coarse propagation runs
  int32_t steps_per_slice; // coarse steps per slice
  int32_t first_sweep;     // 1: k = 0 sweep (no correction)
  double* jump2;           // [samples][M] ||U_new[s] - U_old[s]||^2 (s = slice start index)
  double* norm2;           // [samples][M] ||U[s]||^2
};

// process-wide count of kernels launched by the library
void count_launch(int n = 1);

// ---------------------------------------------------------------- banded direct solver
struct DirectLane {
  const double* LB;        // this lane's band Cholesky factor [n][bw+1]
  const double* invd;      // its reciprocal diagonal [n]
  const double* Binv;      // inverses of its 32 x 32 unit diagonal blocks [n/32][32][32]
  // 64-row blocks of the cluster kernels, [ceil(n/64)][64][64] each:
  const double* B64;       // inverse of the unit lower diagonal block   [b][r][t]
  const double* B64T;      // its transpose                              [b][t][r]
  const double* C1;        // B_b L~_{b,b-1}   column-major [b][t][r]
  const double* C2;        // B_b L~_{b,b-2}   column-major [b][t][r]
  const double* D1;        // L~_{b+1,b} B_b   [b][t][r]
  const double* D2;        // L~_{b+2,b} B_b   [b][t][r]
  const float* LBf;        // FP32 factor, reciprocal diagonal and block inverses (mixed)
  const float* invdf;
  const float* Binvf;
  const double* Av;        // FP64 A values of this lane's sample and dt (mixed residual)
  const double* a_init;    // start state [n] when init_from_a0 (nullptr: start from a0 itself)
  double* b;               // FP64 right-hand side [n] (mixed)
  int32_t* status_out;     // MQS_ST_* bits of this lane (or-ed)
  double *a0, *a1, *y, *w; // lane vectors [n] (lane-major)
  double* qoi_out;         // raw QoI sum of the run, times qoi_scale
  double qoi_scale;        // 1 for the raw sum; 1/T or 1/N to write the finished QoI
  int32_t* done_flag;      // set to 1 (system-wide visible, after qoi_out and status) when
                           // the lane has finished (one-CTA kernels; nullptr: none)
  int64_t vcol;            // value column (sample) of M / K values
  double amp[kMaxPhases], phase[kMaxPhases];
  double dt, t0;
  int64_t k0;              // global index of the first step
  int32_t n_steps, init_from_a0, sample, pad_;
};

struct DirectConst {
  const int32_t* rowptr;
  const int32_t* colidx;
  const int32_t* iperm;    // original -> band ordering
  const int32_t* perm;     // band ordering -> original
  const double* M;         // [nnz][vs] sample values
  const double* K;
  int64_t vs;
  const double* F;         // [P][n]
  int32_t n, bw, n_phases, qoi_kind;
  double omega;
  int32_t w_in_smem;       // 1: the permuted work vector lives in shared memory
  int32_t mixed;           // 1: FP32 factor with FP64 refinement sweeps
  double tol2;             // mixed: stop when ||b - A x||^2 <= tol2 ||b||^2
  int32_t max_sweeps;      // mixed: refinement sweep limit per step
  int32_t cluster;         // 0: one-CTA kernels of mqs_direct.cu; 1, 2, 4, 8: CTAs per lane
  int32_t stall_test;      // 1: the one-CTA cluster kernel's first wait is on a count
                           //    nothing reaches (tests the bounded wait and its status)
  int32_t iter;            // Parareal iteration of this launch (cancellation check)
  // Parareal cancellation (cluster kernels): a launch of iteration `iter`
  // leaves its step loop at the first step boundary where *stop < iter; the
  // word lives in host-mapped memory and is raised by the host once an earlier
  // iteration met the stopping rule (nullptr: never cancelled)
  const volatile int32_t* stop;
};

// One launch of the Parareal coarse sweep of iteration k over slices
// [s_begin, min(s_end, M - 1)).  The sweep starts at slice s_first (k - 1, or
// 0 for k = 0) from U_prev[s_first]; later slices start from U_cur, which it
// writes: U_cur[s + 1] = E[s] + (G_new - G[s]) (Eq. 12), and the jump is
// measured against U_prev[s + 1].  The non-pipelined driver passes one buffer
// as both U_prev and U_cur.
struct DirectChain {
  double *U_prev, *U_cur;  // [samples][M][n] slice starts of iterations k-1 and k
  double *E, *G;           // [samples][M][n] fine ends of iteration k, previous coarse ends
  int32_t M, s_first, s_begin, s_end, steps_per_slice, first_sweep;
  double *jump2, *norm2;   // [samples][M] of iteration k
};

// mqs_api.cu: a context's mesh (nullptr if the id is invalid) and device
const MeshDev* ctx_mesh(mqs_ctx* ctx, int id);
int ctx_device(mqs_ctx* ctx);

// mqs_direct.cu
template <typename T>
int band_factor(const MeshDev& m, const double* A, int64_t vs, int n_fac, T* LB, T* invd, T* Binv,
                int32_t* bad, cudaStream_t st);
int block_count(int n);
int launch_direct(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc, cudaStream_t st);
int direct_smem_max_n(int mixed);
int direct_lane_slots(int mixed);   // -1 on error (message set)
int launch_direct_chain(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                        const DirectChain& ch, cudaStream_t st);

// mqs_cluster.cu: FP64 stepping with the block solve spread over warps and a
// lane split over a cluster of `cluster` CTAs (work vector in shared memory)
int cluster_block_rows();
int band_chol_cluster(double* LB, double* invd, int n, int bw, int64_t fstride, int n_fac,
                      int32_t* bad, cudaStream_t st);
int band_chol_cluster_size();
bool band_chol_cluster_fits(int bw);
int block_prep(const MeshDev& m, int n_fac, const double* LB, double* B, double* BT, double* C1,
               double* C2, double* D1, double* D2, cudaStream_t st);
bool cluster_fits(int n, int bw, int CL);          // own rows + ring fit a CTA's shared memory
int cluster_max_active(int CL, int n, int bw);      // resident clusters (0: does not fit)
int launch_cluster(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc, cudaStream_t st);
int launch_cluster_chain(const DirectLane* d_lanes, int n_lanes, const DirectConst& kc,
                         const DirectChain& ch, cudaStream_t st);

// launchers (mqs_team.cu)
int launch_propagate(const TileDesc* d_tiles, int n_tiles, int L, int C, int precision,
                     const TeamConst& kc, cudaStream_t st);
int launch_chain(const TileDesc* d_tiles, int n_tiles, int L, int C, int precision,
                 const TeamConst& kc, const ChainDesc& ch, cudaStream_t st);
int team_threads();
int max_cluster(int L, int precision, int n_sm);
int max_active_clusters(int L, int precision, int C);

// setup kernels (mqs_setup.cu)
int assemble_region_matrices(MeshDev& m, const double* xy, const int32_t* tri,
                             const int32_t* region, const int32_t* src_phase,
                             const double* src_coef, const std::vector<int32_t>& contrib_ptr,
                             const std::vector<int32_t>& contrib, const std::vector<int32_t>& load_ptr,
                             const std::vector<int32_t>& load, cudaStream_t st);
int expand_values(const MeshDev& m, const double* params, int n_samples, int n_params,
                  double dt, int64_t vs, double* A, double* M, double* K, float* A32,
                  double* Dinv, float* Dinv32, int64_t ds, cudaStream_t st);
int lane_sources(const double* params, int n_samples, int n_params, int n_regions,
                 int n_phases, int lanes_per_sample, double* src_amp, double* src_phi,
                 cudaStream_t st);
int batched_spmv(const MeshDev& m, const double* vals, int64_t vs, int n_samples,
                 const double* x, double* y, cudaStream_t st);

// small kernels (mqs_stats.cu)
int fill_k0(int32_t* k0, int n, int lanes_per_sample, int steps_per_slice, cudaStream_t st);
int copy_lanes(const double* src, double* dst, int64_t n, int64_t xs, int lane_begin,
               int lane_end, int lanes_per_sample, int slice_begin, cudaStream_t st);
int transpose_to_rows(const double* lanes, int64_t xs, int n, int n_samples, int lane_stride,
                      int lane_offset, double* out, cudaStream_t st);
int transpose_from_rows(const double* rows, int n, int n_samples, double* lanes, int64_t xs,
                        cudaStream_t st);
int gather_parareal_qraw(const double* qraw2, int64_t lanes, int M, int K, double* out,
                         cudaStream_t st);
int finish_qoi(const double* raw_fine, const double* raw_coarse, int n_samples, int lanes_per_sample,
               double scale_fine, double scale_coarse, double* qoi, cudaStream_t st);
int mlmc_accumulate_dev(const double* qoi, int n_samples, int level, double* record,
                        cudaStream_t st);

}  // namespace mqs
