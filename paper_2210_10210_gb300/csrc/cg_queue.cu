// Conjugate gradients (Algorithm 2, step 4) for any number of problems of any
// size in one launch, scheduled on the device.
//
// Every problem is a sequence of phases: an initialisation (x = 0, r = p = b,
// ||b||^2), then per iteration the passes of the Toeplitz product (Algorithm 1
// steps 3-6; the first pass also forms p = r + beta p, the last one adds
// sigma^2 p and reduces p^H A p) and the vector update (x += alpha p,
// r -= alpha A p, r^H r).  A phase is split into independent work items (line
// blocks of a pass, chunks of the vectors).  A resident grid of blocks loops:
// it claims an unclaimed item of any problem whose current phase still has
// one (an atomic add on the problem's control word, which carries the phase's
// sequence number, so a claim always knows which phase it belongs to), runs
// it, and counts it complete.  The block completing the last item of a phase
// reduces the items' partial sums in item order (deterministic), updates the
// CG scalars and publishes the next phase.  Problems proceed independently, so
// small problems' short phases fill the gaps between the large ones' and
// nothing waits for a kernel launch.
//
// No block ever waits for a particular other block: a block that finds no
// claimable item polls again (bounded; past the limit it records an error and
// leaves), and blocks leave once every problem has finished.  Hence the
// kernel needs no co-residency guarantee.  Ordering: an item's results are
// released by its completion count (acq_rel), the last completer acquires
// them all, and publishes the next phase with a release store; a claim is an
// acquiring fetch-add, after which the phase's inputs are read with L2-only
// loads.
#include "kernels.h"
#include "line_fft.cuh"

namespace efgp {

constexpr unsigned kSeqDone = 0xffffffffu;
constexpr int kErrQueueIdle = 8;

__device__ __forceinline__ int phase_of(unsigned seq, int npass) {
  return seq == 0 ? 0 : 1 + (int)((seq - 1) % (unsigned)(npass + 1));
}

__device__ __forceinline__ unsigned long long load_word(const unsigned long long* w) {
  return *reinterpret_cast<const volatile unsigned long long*>(w);
}

// claim: fetch-add with acquire semantics (the phase's inputs are read after it)
__device__ __forceinline__ unsigned long long claim_add(unsigned long long* w) {
  unsigned long long old;
  asm volatile("atom.add.acquire.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(w) : "memory");
  return old;
}

// completion count: release the item's results, acquire the others' (last one)
__device__ __forceinline__ unsigned complete_add(unsigned* c) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(c) : "memory");
  return old;
}

// publish the next phase after its scalars
__device__ __forceinline__ void publish(unsigned long long* w, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(w), "l"(v) : "memory");
}

// Runs item `item` of phase `ph`; returns this thread's part of the phase's sum.
// With the Jacobi preconditioner the init and update items also return
// their part of r^H M^-1 r in *s2.
template <typename T>
__device__ double run_item(const QueueProblem& Q, int ph, unsigned item, unsigned char* smem, double* s2) {
  const PersistentProblem& P = Q.P;
  const volatile QueueCtl* c = Q.ctl;
  *s2 = 0.0;
  if (ph == 0 || ph == P.npass + 1) {
    const long long i0 = (long long)item * kQueueChunk;
    const long long i1 = min(P.M, i0 + kQueueChunk);
    double s = 0.0, sz = 0.0;
    if (ph == 0) {
      for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 v = __ldcg(P.b + i);
        const double mi = P.Minv ? P.Minv[i] : 1.0;
        P.x[i] = make_double2(0.0, 0.0);
        P.r[i] = v;
        P.p[i] = make_double2(mi * v.x, mi * v.y);
        const double n2 = v.x * v.x + v.y * v.y;
        s += n2;
        sz += mi * n2;
      }
      *s2 = sz;
    } else {
      const double alpha = c->alpha;
      for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 pv = __ldcg(P.p + i), av = __ldcg(P.Ap + i);
        double2 xv = __ldcg(P.x + i), rv = __ldcg(P.r + i);
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        rv.x -= alpha * av.x;
        rv.y -= alpha * av.y;
        P.x[i] = xv;
        P.r[i] = rv;
        const double n2 = rv.x * rv.x + rv.y * rv.y;
        s += n2;
        if (P.Minv) sz += P.Minv[i] * n2;
      }
      *s2 = sz;
    }
    return s;
  }
  CgArgs cga{};
  cga.Minv = P.Minv;
  cga.src = P.p;
  cga.r = P.r;
  cga.Dw = P.Dw;
  cga.dst = P.Ap;
  cga.sigma2 = P.sigma2;
  cga.update_p = 1;
  return run_pass<T>(P, ph - 1, item, cga, c->beta, smem);
}

// The block that finished phase `ph` (sequence number seq) of problem Q, with
// the phase's total `tot`: CG scalars, then the next phase or the end.
__device__ void advance(const QueueProblem& Q, unsigned seq, int ph, double tot, double tot2, unsigned int* ndone) {
  volatile QueueCtl* c = Q.ctl;
  const PersistentProblem& P = Q.P;
  int done = 0;
  if (ph == 0) {
    c->bnorm2 = tot;
    c->tol2 = P.rho * P.rho * tot;
    c->rr = tot;
    c->rz = P.Minv ? tot2 : tot;
    c->it = 0;
    c->alpha = 0.0;
    c->beta = 0.0;
    if (!isfinite(tot)) done = 3;
    else if (tot == 0.0) done = 1;
    else if (P.max_iter <= 0) done = 2;
  } else if (ph == P.npass) {
    c->pAp = tot;
    if (!(tot > 0.0) || !isfinite(tot)) done = 3;   // breakdown: p^H A p not positive
    else c->alpha = c->rz / tot;
  } else if (ph == P.npass + 1) {
    const long long it = c->it + 1;
    c->it = it;
    const double rz = P.Minv ? tot2 : tot;
    c->beta = rz / c->rz;
    c->rr = tot;
    c->rz = rz;
    if (!isfinite(tot)) done = 3;
    else if (tot <= c->tol2) done = 1;
    else if (it >= P.max_iter) done = 2;
  }
  c->completed = 0u;
  if (done) {
    CgState* st = P.st;
    st->bnorm2 = c->bnorm2;
    st->rr = c->rr;
    st->rr_new = c->rr;
    st->tol2 = c->tol2;
    st->iter = c->it;
    st->max_iter = P.max_iter;
    st->alpha = c->alpha;
    st->beta = c->beta;
    st->pAp = c->pAp;
    st->done = done;
    c->done = done;
    publish(&Q.ctl->word, (unsigned long long)kSeqDone << 32);
    atomicAdd(ndone, 1u);
  } else {
    publish(&Q.ctl->word, (unsigned long long)(seq + 1) << 32);
  }
}

template <typename T>
__global__ void __launch_bounds__(kQueueThreads, sizeof(T) == 4 ? 2 : 1) cg_queue_kernel(const QueueProblem* __restrict__ probs, int nprob,
                                                                 unsigned int* aux, long long idle_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_prob, s_quit, s_last;
  __shared__ unsigned s_seq, s_item;
  unsigned int* ndone = aux;
  int* err = reinterpret_cast<int*>(aux + 1);
  const int tid = threadIdx.x;
  int cursor = blockIdx.x % nprob;
  long long idle = 0;
  for (;;) {
    if (tid < 32) {
      // warp 0 looks for a claimable item, problems taken round-robin from the cursor
      int found = -1;
      unsigned fseq = 0, fitem = 0;
      for (int base = 0; base < nprob && found < 0; base += 32) {
        const int k = base + tid;
        int p = cursor + k;
        if (p >= nprob) p -= nprob;
        bool avail = false;
        if (k < nprob) {
          const unsigned long long w = load_word(&probs[p].ctl->word);
          const unsigned seq = (unsigned)(w >> 32);
          if (seq != kSeqDone) avail = (unsigned)w < (unsigned)probs[p].items[phase_of(seq, probs[p].P.npass)];
        }
        unsigned mask = __ballot_sync(0xffffffffu, avail);
        while (mask && found < 0) {
          const int l = __ffs(mask) - 1;
          mask &= mask - 1;
          int ok = 0;
          unsigned cs = 0, ct = 0;
          if (tid == l) {
            const unsigned long long o = claim_add(&probs[p].ctl->word);
            cs = (unsigned)(o >> 32);
            ct = (unsigned)o;
            ok = cs != kSeqDone && ct < (unsigned)probs[p].items[phase_of(cs, probs[p].P.npass)];
          }
          ok = __shfl_sync(0xffffffffu, ok, l);
          if (ok) {
            found = __shfl_sync(0xffffffffu, p, l);
            fseq = __shfl_sync(0xffffffffu, cs, l);
            fitem = __shfl_sync(0xffffffffu, ct, l);
          }
        }
      }
      if (tid == 0) {
        s_prob = found;
        s_seq = fseq;
        s_item = fitem;
        s_quit = found < 0 && *reinterpret_cast<volatile unsigned int*>(ndone) >= (unsigned)nprob;
      }
    }
    __syncthreads();
    const int pi = s_prob;
    if (s_quit) break;
    if (pi < 0) {
      if (++idle > idle_limit) {
        if (tid == 0) atomicOr(err, kErrQueueIdle);
        break;
      }
      __nanosleep(64);
      __syncthreads();
      continue;
    }
    idle = 0;
    cursor = pi + 1 == nprob ? 0 : pi + 1;
    const QueueProblem& Q = probs[pi];
    const unsigned seq = s_seq, item = s_item;
    const int npass = Q.P.npass;
    const int ph = phase_of(seq, npass);
    double part2 = 0.0;
    const double part = run_item<T>(Q, ph, item, smem_raw, &part2);
    const bool reduce = ph == 0 || ph == npass || ph == npass + 1;
    const bool reduce2 = Q.P.Minv && (ph == 0 || ph == npass + 1);
    double bs = 0.0, bs2 = 0.0;
    if (reduce) bs = block_sum(part, red);
    if (reduce2) {
      __syncthreads();
      bs2 = block_sum(part2, red);
    }
    if (tid == 0) {
      if (reduce) Q.partials[item] = bs;
      if (reduce2) Q.partials2[item] = bs2;
      const unsigned done_items = complete_add(&Q.ctl->completed);
      s_last = done_items == (unsigned)Q.items[ph] - 1;
    }
    __syncthreads();
    if (s_last) {
      double tot = 0.0, tot2 = 0.0;
      if (reduce) tot = block_sum_partials(Q.partials, Q.items[ph], red);
      if (reduce2) {
        __syncthreads();
        tot2 = block_sum_partials(Q.partials2, Q.items[ph], red);
      }
      if (tid == 0) advance(Q, seq, ph, tot, tot2, ndone);
    }
    __syncthreads();
  }
}

template <typename T>
static cudaError_t launch_t(const QueueProblem* d_probs, int nprob, unsigned int* aux, size_t smem, int blocks,
                            long long idle_limit, cudaStream_t s) {
  auto kern = cg_queue_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kQueueThreads, smem, s>>>(d_probs, nprob, aux, idle_limit);
  return cudaGetLastError();
}

cudaError_t launch_cg_queue(const QueueProblem* d_probs, int nprob, unsigned int* aux, int f64, size_t smem,
                            int blocks, long long idle_limit, cudaStream_t s) {
  return f64 ? launch_t<double>(d_probs, nprob, aux, smem, blocks, idle_limit, s)
             : launch_t<float>(d_probs, nprob, aux, smem, blocks, idle_limit, s);
}

int cg_queue_blocks(int f64, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e;
  if (f64) {
    cudaFuncSetAttribute(cg_queue_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cg_queue_kernel<double>, kQueueThreads, smem);
  } else {
    cudaFuncSetAttribute(cg_queue_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cg_queue_kernel<float>, kQueueThreads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * sms;
}

}  // namespace efgp
