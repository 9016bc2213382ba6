// efgp_predict_noalloc: the posterior mean at targets without allocating.
//
// Some callers cannot allocate device memory at the point where they need
// predictions: real-time serving loops that must not block in the allocator,
// and host applications that reserve all device memory up front and forbid
// plug-ins from allocating.  This entry point serves them: it runs the same
// type-2 steps as efgp_predict, but its two scratch grids live in one
// statically sized device array defined in this file instead of handle
// memory allocated on first use.  Like efgp_predict it ends with a read-back
// of the target range flag and a synchronisation of the handle's stream.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "handle.h"
#include "kernels.h"

// Largest scratch the entry point can use: the type-2 fine grid (complex)
// plus the extended real grid.  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the array, looked up once per device (in host code the
// array's name is only a host-side stand-in and must not be passed to a kernel).
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    efgp::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return EFGP_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    efgp::set_error("device index out of range");
    return EFGP_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      efgp::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return EFGP_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return EFGP_OK;
}

long long ipow_n(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

#define NA_CK(call)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      efgp::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));           \
      return EFGP_ECUDA;                                                             \
    }                                                                                \
  } while (0)

}  // namespace

extern "C" int efgp_predict_noalloc(efgp_handle* H, const void* targets, int64_t q, void* mu_out) {
  if (!H) return EFGP_EINVAL;
  if (!H->solved) {
    efgp::set_error("efgp_predict_noalloc before efgp_solve");
    return EFGP_ESTATE;
  }
  if (H->opt.host_io) {
    efgp::set_error("efgp_predict_noalloc takes device pointers only (host_io handles need staging buffers)");
    return EFGP_EINVAL;
  }
  if (q < 0 || (q > 0 && (!targets || !mu_out))) return EFGP_EINVAL;
  if (q == 0) return EFGP_OK;
  const int d = H->d;
  const efgp::NufftPlan& p2 = H->p2;
  const long long nf_tot = ipow_n(p2.nf, d);
  const long long nE_tot = ipow_n(p2.nE, d);
  // fine grid first, extended real grid after it at a 256-byte boundary
  const size_t g_bytes = H->elem * (size_t)nf_tot;
  const size_t e_off = (g_bytes + 255) & ~(size_t)255;
  const size_t need = e_off + (H->f64 ? 8 : 4) * (size_t)nE_tot;
  if (need > kNoAllocScratchBytes) {
    efgp::set_error("efgp_predict_noalloc: this problem's type-2 grids need " + std::to_string(need) +
                    " bytes of scratch, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
                    "; use efgp_predict");
    return EFGP_EUNSUPPORTED;
  }
  void* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != EFGP_OK) return rc;
  void* g2 = base;
  void* E2 = static_cast<unsigned char*>(base) + e_off;
  const int coord_f64 = H->opt.coord_dtype == EFGP_F64;
  const int value_f64 = H->opt.value_dtype == EFGP_F64;
  // the array keeps the previous call's contents: the fine grid must start at
  // zero (the extended grid is overwritten in full by the unfold)
  NA_CK(cudaMemsetAsync(g2, 0, g_bytes, H->stream));
  NA_CK(cudaMemsetAsync(H->flag, 0, sizeof(int), H->stream));
  NA_CK(efgp::launch_precorrect(H->x, H->Dw, H->corr2, H->par.m, d, p2.nf, g2, H->f64, H->stream));
  const int frc = efgp::internal_grid_fft(H, p2.nf, +1, g2, H->f64, H->twF2);
  if (frc != EFGP_OK) return frc;
  NA_CK(efgp::launch_unfold(g2, H->f64, p2.nf, d, p2.off, p2.nE, E2, H->stream));
  const efgp::GridScale gs = efgp::internal_make_scale(p2);
  const void* coef = H->f64 ? (const void*)&H->c2d : (const void*)&H->c2f;
  NA_CK(efgp::launch_interp(targets, coord_f64, H->opt.x_layout == 1, q, d, p2.w, gs, p2.off, p2.nE, E2, H->f64, coef,
                            mu_out, value_f64, H->flag, H->stream));
  H->times.launches += 3;
  NA_CK(cudaMemcpyAsync(H->host_flag, H->flag, sizeof(int), cudaMemcpyDeviceToHost, H->stream));
  NA_CK(cudaStreamSynchronize(H->stream));
  if (*H->host_flag) {
    efgp::set_error("a target lies outside [0,1] or is not finite");
    return EFGP_ERANGE;
  }
  return EFGP_OK;
}
