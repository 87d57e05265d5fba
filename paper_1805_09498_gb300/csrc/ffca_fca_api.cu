// C ABI of the conventional FCA EM baseline (Sec. 3.3).  See include/ffca.h.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "ffca.h"
#include "ffca_dispatch.h"
#include "ffca_fca.cuh"

using namespace ffca;

namespace ffca {

const FcaKernels* fca_kernels(int prec, int I, int J) {
  if (prec == 0) {
    switch (I) {
      case 1: return fca_kernels_p0_i1(J);
      case 2: return fca_kernels_p0_i2(J);
      case 3: return fca_kernels_p0_i3(J);
      case 4: return fca_kernels_p0_i4(J);
      case 8: return fca_kernels_p0_i8(J);
    }
  } else if (prec == 1) {
    switch (I) {
      case 1: return fca_kernels_p1_i1(J);
      case 2: return fca_kernels_p1_i2(J);
      case 3: return fca_kernels_p1_i3(J);
      case 4: return fca_kernels_p1_i4(J);
      case 8: return fca_kernels_p1_i8(J);
    }
  }
  return nullptr;
}

}  // namespace ffca

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr int kFinalThreads = 128;

struct FcaPlan {
  Partition p;
  size_t off_llf, off_trace, off_tab, off_part, bytes;
};

ffca_status fca_check_shape(const ffca_fca_desc* d) {
  if (!d) return FFCA_ERR_ARG;
  if (d->prec != FFCA_PREC_FP64 && d->prec != FFCA_PREC_MIXED) return FFCA_ERR_ARG;
  if (d->F < 0 || d->N < 1 || d->ld < d->N || (d->ld % 4) != 0) return FFCA_ERR_ARG;
  if (d->I < 1 || d->J < 1) return FFCA_ERR_ARG;
  if ((d->I > 4 && d->I != 8) || d->J > 6) return FFCA_ERR_UNSUPPORTED;
  return FFCA_OK;
}

ffca_status fca_plan(const ffca_fca_desc* d, const FcaKernels* k, FcaPlan* p) {
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FFCA_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FFCA_ERR_CUDA;
  if (k->em_smem > 0)
    for (const void* fn : {k->em_update, k->em_eval})
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->em_smem) != cudaSuccess)
        return FFCA_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->em_update, kBlock, k->em_smem) != cudaSuccess)
    return FFCA_ERR_CUDA;
  if (occ < 1) return FFCA_ERR_INTERNAL;
  const int FU = d->prec == FFCA_PREC_FP64 ? 1 : 2;
  const int F = d->F > 0 ? d->F : 1;
  p->p = make_partition(F, (d->N + FU - 1) / FU, nsm * occ);
  p->p.F = d->F;
  const int NV = k->nv;
  size_t off = kAlign;  // status words, counter, operation counts
  p->off_llf = off; off = align_up(off + sizeof(double) * F);
  p->off_trace = off; off = align_up(off + sizeof(double) * kTraceCap);
  p->off_tab = off; off = align_up(off + (size_t)F * k->params_bytes);
  p->off_part = off; off = align_up(off + sizeof(double) * (size_t)F * p->p.max_slots * NV);
  p->bytes = off;
  return FFCA_OK;
}

}  // namespace

struct ffca_fca_ctx {
  ffca_fca_desc d;
  const FcaKernels* k;
  FcaPlan plan;
  cudaStream_t stream;
  char* ws;
  int err_f;
};

namespace {

FcaArgs fca_args(const ffca_fca_ctx* c, int slot) {
  FcaArgs a;
  std::memset(&a, 0, sizeof(a));
  a.part = c->plan.p;
  a.F = c->d.F;
  a.N = c->d.N;
  a.ld = c->d.ld;
  a.y = c->d.y;
  a.v = c->d.v;
  a.S = c->d.S;
  a.tab = c->ws + c->plan.off_tab;
  a.part_buf = reinterpret_cast<double*>(c->ws + c->plan.off_part);
  a.llf = reinterpret_cast<double*>(c->ws + c->plan.off_llf);
  a.trace = reinterpret_cast<double*>(c->ws + c->plan.off_trace);
  a.trace_slot = slot;
  a.status = reinterpret_cast<unsigned*>(c->ws);
  a.gcnt = reinterpret_cast<unsigned*>(c->ws + 16);
  a.ops = reinterpret_cast<unsigned long long*>(c->ws + 32);
  a.mults = reinterpret_cast<unsigned long long*>(c->ws + 40);
  a.inv_n = 1.0 / c->d.N;
  return a;
}

ffca_status fca_launch(const ffca_fca_ctx* c, const void* fn, int grid, int block, FcaArgs& a, size_t smem = 0) {
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, c->stream) == cudaSuccess ? FFCA_OK
                                                                                             : FFCA_ERR_CUDA;
}

// one thread per frequency (small arrays) or one warp per frequency (I > 4)
int fca_final_grid(const ffca_fca_ctx* c) {
  const int per_block = c->k->final_block == 1 ? kFinalThreads : kFinalThreads / 32;
  return (c->d.F + per_block - 1) / per_block;
}

ffca_status fca_status(ffca_fca_ctx* c) {
  unsigned h[2] = {0, 0};
  if (cudaMemcpyAsync(h, c->ws, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  c->err_f = h[0] ? (int)h[1] : -1;
  return (ffca_status)h[0];
}

// log-likelihood-only pass of the current state into trace slot `slot`
ffca_status fca_eval(ffca_fca_ctx* c, int slot) {
  FcaArgs a = fca_args(c, slot);
  ffca_status st = fca_launch(c, c->k->em_eval, a.part.nblocks, kBlock, a, c->k->em_smem);
  if (st != FFCA_OK) return st;
  return fca_launch(c, c->k->final_eval, fca_final_grid(c), kFinalThreads, a);
}

}  // namespace

extern "C" {

size_t ffca_fca_workspace_size(const ffca_fca_desc* d) {
  if (fca_check_shape(d) != FFCA_OK) return 0;
  const FcaKernels* k = fca_kernels(d->prec, d->I, d->J);
  if (!k) return 0;
  FcaPlan p;
  if (fca_plan(d, k, &p) != FFCA_OK) return 0;
  return p.bytes;
}

ffca_status ffca_fca_init(ffca_fca_ctx** out, const ffca_fca_desc* d) {
  if (!out) return FFCA_ERR_ARG;
  *out = nullptr;
  ffca_status st = fca_check_shape(d);
  if (st != FFCA_OK) return st;
  if (d->F > 0) {
    auto al = [](const void* p, uintptr_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) == 0; };
    if (!al(d->y, 16) || !al(d->v, 16) || !al(d->S, 16) || !al(d->workspace, kAlign)) return FFCA_ERR_ARG;
  }
  const FcaKernels* k = fca_kernels(d->prec, d->I, d->J);
  if (!k) return FFCA_ERR_UNSUPPORTED;
  FcaPlan p;
  if ((st = fca_plan(d, k, &p)) != FFCA_OK) return st;
  if (d->F > 0 && d->workspace_bytes < p.bytes) return FFCA_ERR_ARG;
  ffca_fca_ctx* c = static_cast<ffca_fca_ctx*>(std::calloc(1, sizeof(ffca_fca_ctx)));
  if (!c) return FFCA_ERR_INTERNAL;
  c->d = *d;
  c->k = k;
  c->plan = p;
  c->stream = static_cast<cudaStream_t>(d->stream);
  c->ws = static_cast<char*>(d->workspace);
  c->err_f = -1;
  if (d->F > 0 && cudaMemsetAsync(c->ws, 0, p.bytes, c->stream) != cudaSuccess) {
    std::free(c);
    return FFCA_ERR_CUDA;
  }
  *out = c;
  return FFCA_OK;
}

ffca_status ffca_fca_iterate(ffca_fca_ctx* c, int iters, double* ll_trace) {
  if (!c || iters < 0) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    if (ll_trace)
      for (int t = 0; t <= iters; ++t) ll_trace[t] = 0.0;
    return FFCA_OK;
  }
  FcaArgs a0 = fca_args(c, 0);
  ffca_status st = fca_launch(c, c->k->prep, (c->d.F + 127) / 128, 128, a0);
  if (st != FFCA_OK) return st;
  const double* dtrace = reinterpret_cast<const double*>(c->ws + c->plan.off_trace);
  int flushed = 0;
  for (int t = 0; t <= iters; ++t) {
    const int slot = t % kTraceCap;
    if (t < iters) {
      FcaArgs a = fca_args(c, slot);
      if ((st = fca_launch(c, c->k->em_update, a.part.nblocks, kBlock, a, c->k->em_smem)) != FFCA_OK) return st;
      if ((st = fca_launch(c, c->k->final_update, fca_final_grid(c), kFinalThreads, a)) != FFCA_OK) return st;
    } else if (ll_trace) {
      if ((st = fca_eval(c, slot)) != FFCA_OK) return st;
    }
    if (ll_trace && (slot == kTraceCap - 1 || t == iters)) {
      const int n = t - flushed + 1;
      if (cudaMemcpyAsync(ll_trace + flushed, dtrace, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess)
        return FFCA_ERR_CUDA;
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
      flushed = t + 1;
    }
  }
  if (ll_trace) return fca_status(c);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

ffca_status ffca_fca_loglik(ffca_fca_ctx* c, double* ll) {
  if (!c || !ll) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    *ll = 0.0;
    return FFCA_OK;
  }
  FcaArgs a0 = fca_args(c, 0);
  ffca_status st = fca_launch(c, c->k->prep, (c->d.F + 127) / 128, 128, a0);
  if (st != FFCA_OK) return st;
  if ((st = fca_eval(c, 0)) != FFCA_OK) return st;
  if (cudaMemcpyAsync(ll, c->ws + c->plan.off_trace, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return FFCA_ERR_CUDA;
  return fca_status(c);
}

ffca_status ffca_fca_op_counts(ffca_fca_ctx* c, unsigned long long* inversions,
                               unsigned long long* multiplications) {
  if (!c) return FFCA_ERR_ARG;
  unsigned long long h[2] = {0, 0};
  if (c->d.F > 0) {
    if (cudaMemcpyAsync(h, c->ws + 32, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return FFCA_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  }
  if (inversions) *inversions = h[0];
  if (multiplications) *multiplications = h[1];
  return FFCA_OK;
}

int ffca_fca_error_frequency(const ffca_fca_ctx* c) { return c ? c->err_f : -1; }

void ffca_fca_destroy(ffca_fca_ctx* c) { std::free(c); }

}  // extern "C"
