// Internal definition of the problem handle, shared by the translation
// units that implement the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.h"

namespace efgp {

// One pass of a multi-axis FFT or of the Toeplitz product.
struct Pass {
  LineGeom g;
  int in_buf;   // buffer ids, interpreted by the caller
  int out_buf;
  int dir;
  int inm, outm;
  bool conv;
  int threads;
  int kind = 0;   // 0 line batches; 1, 2: forward, inverse plane pass of the 3D product
  int n1 = 0;     // plane passes: data extent per axis
};

bool fault_injected(const char* what);

}  // namespace efgp

using efgp::CgState;
using efgp::EsCoef;
using efgp::NufftPlan;
using efgp::Pass;

struct efgp_handle {
  int d = 0;
  long long N = 0;
  efgp_kernel kern{};
  double sigma = 0, eps = 0;
  efgp_options opt{};
  efgp_params par{};
  NufftPlan p1, p2;
  int f64 = 0;          // FP64 Toeplitz products, CG grids and type-2 grids
  int sf64 = 0;         // FP64 spread and fine grid of the set-up (plain precision)
  size_t elem = 8;      // bytes of one complex grid element
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  long long M = 0;
  int n1 = 0;
  // device arrays
  double* Dw = nullptr;
  double* corr1 = nullptr;
  double* corr2 = nullptr;
  double2* w = nullptr;
  double2* b = nullptr;
  void* what = nullptr;
  void* twL = nullptr;
  void* twF2 = nullptr;
  double2 *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr;
  CgState* st = nullptr;
  double* partials = nullptr;
  double* Minv = nullptr;   // Jacobi preconditioner (options.precond)
  void* scrA = nullptr;
  void* scrB = nullptr;
  void* g2 = nullptr;
  void* E2 = nullptr;
  int* flag = nullptr;
  double* dsum = nullptr;
  unsigned int* ticket = nullptr;
  CgState* host_state = nullptr;
  int* host_flag = nullptr;
  char* pinned = nullptr;   // 256-byte pinned slot holding host_state and host_flag
  // plans
  std::vector<Pass> mv;
  std::vector<Pass> mvg;   // the product as captured in the CG graph (3D: plane passes where they fit)
  std::vector<Pass> fft2;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  EsCoef<float> c1f{}, c2f{};
  EsCoef<double> c1d{}, c2d{};
  bool solved = false;
  bool tuned = false;       // options.autotune applied to the Toeplitz passes
  std::vector<void*> allocs;
  efgp_phase_times times{};
  // persistent CG (one launch on a thread-block cluster)
  int pcluster = -1;                    // -1 undecided, 0 not eligible, else cluster size
  size_t psmem = 0;
  efgp::PersistentProblem pprob{};
  efgp::PersistentProblem* d_pprob = nullptr;
  // persistent CG over the whole GPU (cg_grid.cu)
  int gblocks = -1;                     // -1 undecided, 0 not eligible, else blocks of the launch
  size_t gsmem = 0;
  efgp::PersistentProblem gprob{};
  efgp::PersistentProblem* d_gprob = nullptr;
  efgp::GridBarrier* gbar = nullptr;
  double* gpart = nullptr;
  // dynamically scheduled CG (cg_queue.cu)
  double* qpartials = nullptr;
  long long qpartials_n = 0;
  efgp::QueueCtl* qctl = nullptr;
  efgp::QueueProblem* d_qprob = nullptr;
  unsigned int* qaux = nullptr;
  cudaEvent_t ev[8] = {};
  bool ev_made = false;

  void mark(int i) {
    if (!opt.profile) return;
    if (!ev_made) {
      for (auto& e : ev) cudaEventCreate(&e);
      ev_made = true;
    }
    cudaEventRecord(ev[i], stream);
  }
  double span(int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[a], ev[b]) != cudaSuccess) return 0.0;
    return ms;
  }

  int alloc(void** ptr, size_t bytes) {
    if (efgp::fault_injected("alloc")) {
      efgp::set_error("injected allocation failure (EFGP_FAULT=alloc)");
      return EFGP_ENOMEM;
    }
    if (bytes == 0) bytes = 16;
    // stream-ordered allocation from the device pool: cheap to repeat for
    // every set-up, and released without a device-wide synchronisation
    cudaError_t e = cudaMallocAsync(ptr, bytes, stream);
    if (e != cudaSuccess) {
      efgp::set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? EFGP_ENOMEM : EFGP_ECUDA;
    }
    allocs.push_back(*ptr);
    return EFGP_OK;
  }
};

namespace efgp {
// FFT of a full n^d grid in place (dir -1 forward, +1 inverse).
int internal_grid_fft(efgp_handle* H, int n, int dir, void* grid, bool f64, const void* tw);
GridScale internal_make_scale(const NufftPlan& p);
}  // namespace efgp
