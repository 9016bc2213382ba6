// Host-callable launchers of the CUDA kernels of libefgp.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace efgp {

// Arguments of the CG-aware first (prologue) and last (epilogue) passes of
// the Toeplitz matrix-vector product.
struct CgArgs {
  double2* src;          // vector the operator is applied to (p in CG)
  const double2* r;      // residual (for the p update)
  const double* Dw;      // spectral weights D (M)
  double2* dst;          // output (A src)
  double sigma2;         // sigma^2
  CgState* st;           // CG scalars (may be null outside CG)
  double* partials;      // per-block partial dot products
  const double* Minv;    // Jacobi preconditioner 1 / diag(A) (M), or null (plain CG)
  int update_p;          // 1: first pass sets src = r + beta*src (iteration > 0)
  int do_dot;            // 1: last pass reduces Re(src^H dst) into st->pAp, alpha
  int check_done;        // 1: skip everything once st->done is set
};

enum LineIn { IN_PLAIN = 0, IN_CG = 1 };
enum LineOut { OUT_PLAIN = 0, OUT_CG = 1 };

// One batched pass of length-L FFTs along one axis (see LineGeom).  dir = -1
// forward, +1 inverse (unnormalised).  With what != nullptr the pass is a
// forward FFT, a pointwise product with the real array what (index
// (o*L + k)*inner + i) and an inverse FFT.
template <typename T>
cudaError_t launch_line_fft(const LineGeom& g, const void* in, void* out, int dir, const cplx<T>* tw, const T* what,
                            int inm, int outm, const CgArgs* cga, int threads, cudaStream_t s);

size_t line_fft_smem_bytes(int L, int nb, size_t elem_bytes);

// 3D Toeplitz product, inner two axes per slab (one block per j0 < n1): the
// forward pass reads the CG vector (prologue) and writes S [n1][L][L]; the
// inverse pass reads S and applies the CG epilogue and reduction.
constexpr int kPlaneThreads = 512;
size_t plane_fft_smem_bytes(int L, size_t elem_bytes);
template <typename T>
cudaError_t launch_plane_fft(const LineGeom& g, int n1, int inverse, void* S, const cplx<T>* tw, const CgArgs& cga,
                             cudaStream_t s);
template <typename T>
cudaError_t prepare_plane_fft();
constexpr int kLineFftMaxSmem = 200 * 1024;   // dynamic shared memory cap of one pass
constexpr size_t kLineFftBlockSmem = 100 * 1024;   // preferred cap (two blocks per SM)
constexpr int kLineFftMaxThreads = 512;
constexpr int kMaxLineBatch = 32;   // lines of one block (per-line offset table in shared memory)
template <typename T>
cudaError_t prepare_line_fft();

// ---- persistent CG on one thread-block cluster per problem (cg_persistent.cu)
constexpr int kMaxPasses = 5;
constexpr int kPersistentThreads = 256;
struct PersistentProblem {
  LineGeom pass[kMaxPasses];
  int npass;
  int inb[kMaxPasses], outb[kMaxPasses], dir[kMaxPasses], inm[kMaxPasses], outm[kMaxPasses], conv[kMaxPasses];
  void* buf[3];          // buffer ids of the passes: 0 unused, 1 and 2 scratch
  const void* tw;        // twiddles of length L (grid precision)
  const void* what;      // transformed generating vector (grid precision)
  double2 *x, *r, *p, *Ap;
  const double2* b;
  const double* Dw;
  double sigma2;
  long long M;
  double rho;
  long long max_iter;
  CgState* st;           // final state written here
  const double* Minv;    // Jacobi preconditioner (scheduled CG), or null
};
cudaError_t launch_cg_persistent(const PersistentProblem* d_probs, int nprob, int cluster, size_t smem, int f64,
                                 cudaStream_t s);
int persistent_cluster_size(int f64, size_t smem);

// ---- persistent CG on the whole GPU, one cooperative launch (cg_grid.cu)
constexpr int kGridCgThreads = 256;
// Grid barrier state (host zeroes it before every launch).
struct GridBarrier {
  unsigned int count;   // blocks arrived at the current barrier
  unsigned int gen;     // barriers completed
  int err;              // non-zero: a block gave up waiting
  int pad;
};
constexpr long long kGridWaitLimit = 1ll << 24;   // polls of one barrier wait (seconds)
// part: 2 * blocks doubles of per-block partial sums
cudaError_t launch_cg_grid(const PersistentProblem* d_prob, GridBarrier* gb, double* part, int blocks, size_t smem,
                           int f64, long long limit, cudaStream_t s);
int cg_grid_blocks(int f64, size_t smem);   // blocks of the cooperative launch (0: not possible)

// ---- dynamically scheduled CG over many problems in one launch (cg_queue.cu)
constexpr int kQueueThreads = 512;
constexpr int kQueueChunk = 2048;   // vector elements per item of the init and update phases
// Control block of one problem, in global memory, one cache line each.
struct alignas(128) QueueCtl {
  unsigned long long word;   // (phase sequence number << 32) | items claimed in it
  unsigned int completed;    // items of the current phase finished
  int done;                  // 0 running, 1 converged, 2 iteration cap, 3 breakdown
  double rr, alpha, beta, bnorm2, tol2, pAp;
  long long it;
  double rz;                 // r^H M^-1 r (= rr without a preconditioner)
};
struct QueueProblem {
  PersistentProblem P;           // passes (line batches chosen for this kernel), buffers, scalars
  int items[kMaxPasses + 2];     // work items of phase 0 (init), 1..npass (passes), npass+1 (update)
  double* partials;              // one partial sum per item of the largest phase
  double* partials2;             // second sums of the init and update items (r^H z), or null
  QueueCtl* ctl;
};
// aux[0]: problems finished, aux[1]: error flags (host zeroes both and every
// ctl).  A block that finds nothing to claim idle_limit times in a row sets an
// error flag and returns.
constexpr long long kQueueIdleLimit = 1ll << 24;   // ~10 s of empty polls
cudaError_t launch_cg_queue(const QueueProblem* d_probs, int nprob, unsigned int* aux, int f64, size_t smem,
                            int blocks, long long idle_limit, cudaStream_t s);
int cg_queue_blocks(int f64, size_t smem);   // resident blocks of the kernel on the device (0: does not fit)

// Launch `kern` with programmatic stream serialisation (the next kernel in the
// stream may be scheduled before this one finishes; kernels that are launched
// this way call grid_dependency_wait() first).
template <typename K, typename... Args>
cudaError_t launch_pdl(K kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- CG vector kernels (cg.cu)
// Minv: the Jacobi preconditioner 1 / diag(A), or null for plain CG.
cudaError_t launch_cg_init(const double2* b, double2* x, double2* r, double2* p, long long M, double rho,
                           long long max_iter, CgState* st, double* partials, const double* Minv, cudaStream_t s);
cudaError_t launch_cg_update(double2* x, double2* r, const double2* p, const double2* Ap, long long M, CgState* st,
                             double* partials, const double* Minv, cudaStream_t s);
// Minv_j = 1 / (D_j^2 Re w_0 + sigma^2): the diagonal of D W D + sigma^2 I
cudaError_t launch_jacobi(const double* Dw, const double2* w_center, double sigma2, long long M, double* Minv,
                          cudaStream_t s);
cudaError_t launch_residual_norm(const double2* b, const double2* Ax, long long M, double* out_sum, double* partials,
                                 unsigned int* ticket, cudaStream_t s);
int cg_blocks(long long M);

// ---- setup kernels (spread.cu and friends)
struct SortGeom {
  GridScale gs;
  int d;
  int W;
  int off;          // extended-grid offset
  int TB;           // tile edge
  int nt[3];        // tiles per dim
  int ntiles;
  int nEx;          // extended grid per dim (nt*TB + W - 1)
  int x_vec;        // 1: row-major 2D float coordinates are 8-byte aligned (vector loads)
  long long rstride;  // elements between the sorted record arrays (>= N + 4, multiple of 4)
};

cudaError_t launch_bin_count(const void* x, int coord_f64, int rec_f64, int soa, long long N, const SortGeom& sg,
                             unsigned int* counts, int* range_flag, cudaStream_t s);
cudaError_t launch_scan_tiles(const unsigned int* counts, int ntiles, long long* tile_off, long long* cursor,
                              cudaStream_t s);
cudaError_t launch_bin_scatter(const void* x, int coord_f64, const void* y, int value_f64, int soa, long long N,
                               const SortGeom& sg, int rec_f64, long long* cursor, void* rec, int* err, cudaStream_t s);
cudaError_t launch_spread(const void* rec, int rec_f64, long long N, const SortGeom& sg, const long long* tile_off,
                          const void* coef, double2* E, int* err, cudaStream_t s);
cudaError_t launch_spectral_weights(double* Dw, int m, int d, double h, const efgp_kernel& k, cudaStream_t s);
cudaError_t launch_fold(const double2* E, int nEx, int off, int nf, int d, void* P, int p_f64, cudaStream_t s);
cudaError_t launch_deconv_split(const void* Phat, int p_f64, int nf, int d, int m, const double* corr1,
                                const double* Dw, double2* w, double2* b, cudaStream_t s);
cudaError_t launch_place_w(const double2* w, int m, int d, int L, double2* grid, cudaStream_t s);
cudaError_t launch_extract_what(const double2* grid, long long n, double scale, void* what, int what_f64,
                                cudaStream_t s);

// ---- fused chunked set-up, 2D FP32 points (setup_fused.cu)
constexpr int kFusedMaxTiles = 1024;   // spread tiles of the fused path (shared-memory histograms)
constexpr int kFusedMaxWidth = 6;      // ES widths whose W x W register footprint fits
// FP64 accumulator of one cell of a halo'd tile: sums and compensations.
struct alignas(32) TileAcc {
  double sx, sy, cx, cy;
};
struct FusedArgs {
  const float* x;               // N x 2 row-major, 16-byte aligned
  const float* y;               // N, 16-byte aligned
  long long N;
  SortGeom sg;
  long long share;              // points of one block's share of a chunk (multiple of 4096)
  long long chunk;              // points per chunk = blocks * share
  int nchunks;
  const unsigned int* off;      // [nchunks][blocks][ntiles]: chunk position of a share's first point per tile
  const unsigned int* toff;     // [nchunks][ntiles + 1]: first chunk position of each tile
  float* B[2];                  // chunk buffers (k mod 2): arrays q0, q1, y of bstride floats each
  long long bstride;            // >= chunk + 8, multiple of 4
  float2* slots[2];             // tile-visit partials of chunk k mod 2: (blocks + ntiles) x S^2
  TileAcc* Et;                  // ntiles x S^2 halo'd tiles (sums and compensations)
};
size_t fused_smem_bytes(int ntiles, int W);
int fused_blocks(int W, size_t smem);   // resident blocks of the cooperative launch (0: not possible)
cudaError_t launch_fused_count(const float* x, long long N, const SortGeom& sg, long long share, long long chunk,
                               int blocks, int nchunks, unsigned int* cnt, int* range_flag, cudaStream_t s);
cudaError_t launch_tile_totals_2d(const float* x, long long N, const SortGeom& sg, unsigned int* counts,
                                  int* range_flag, cudaStream_t s);
cudaError_t launch_fused_scan(unsigned int* cnt, int blocks, int ntiles, int nchunks, unsigned int* toff,
                              cudaStream_t s);
cudaError_t launch_setup_fused(const FusedArgs& a, const void* coef, int blocks, size_t smem, GridBarrier* gb,
                               long long limit, int* err, cudaStream_t s);
cudaError_t launch_fused_fold(const TileAcc* Et, const SortGeom& sg, int nf, int off, float2* P, cudaStream_t s);

// ---- predict kernels (interp.cu)
cudaError_t launch_precorrect(const double2* beta, const double* Dw, const double* corr2, int m, int d, int nf,
                              void* g, int g_f64, cudaStream_t s);
cudaError_t launch_unfold(const void* g, int g_f64, int nf, int d, int off, int nE, void* E2, cudaStream_t s);
cudaError_t launch_interp(const void* targets, int coord_f64, int soa, long long q, int d, int W, const GridScale& gs,
                          int off, int nE, const void* E2, int g_f64, const void* coef, void* mu, int value_f64,
                          int* range_flag, cudaStream_t s);

}  // namespace efgp
