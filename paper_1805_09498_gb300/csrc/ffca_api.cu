// C ABI of the FastFCA-AS library: validation, launch planning, workspace
// carving and the per-iteration launch sequence.  See include/ffca.h.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ffca.h"
#include "ffca_adjoint.cuh"
#include "ffca_dispatch.h"
#include "ffca_mask.cuh"
#include "ffca_resident.cuh"
#include "ffca_stream.cuh"

using namespace ffca;

namespace ffca {

const FastKernels* fast_kernels(int prec, int I, int J) {
  if (prec == 0) {
    switch (I) {
      case 1: return fast_kernels_p0_i1(J);
      case 2: return fast_kernels_p0_i2(J);
      case 3: return fast_kernels_p0_i3(J);
      case 4: return fast_kernels_p0_i4(J);
      case 8: return fast_kernels_p0_i8(J);
    }
  } else if (prec == 1) {
    switch (I) {
      case 1: return fast_kernels_p1_i1(J);
      case 2: return fast_kernels_p1_i2(J);
      case 3: return fast_kernels_p1_i3(J);
      case 4: return fast_kernels_p1_i4(J);
      case 8: return fast_kernels_p1_i8(J);
    }
  }
  return nullptr;
}

const AdjKernels* adj_kernels(int prec, int I, int J) {
  if (prec == 0) {
    switch (I) {
      case 1: return adj_kernels_p0_i1(J);
      case 2: return adj_kernels_p0_i2(J);
      case 3: return adj_kernels_p0_i3(J);
      case 4: return adj_kernels_p0_i4(J);
      case 8: return adj_kernels_p0_i8(J);
    }
  } else if (prec == 1) {
    switch (I) {
      case 1: return adj_kernels_p1_i1(J);
      case 2: return adj_kernels_p1_i2(J);
      case 3: return adj_kernels_p1_i3(J);
      case 4: return adj_kernels_p1_i4(J);
      case 8: return adj_kernels_p1_i8(J);
    }
  }
  return nullptr;
}

}  // namespace ffca

namespace {

constexpr size_t kAlign = 256;

// Candidate partitions of a batch (ffca_batch_autotune): the fixed cost per
// problem segment the CTA ranges balance, in frames of streaming work, and
// the grid size in waves of resident CTAs.  Candidate 0 is the default: the
// segment costs measured on GB300 for the batched workload's shapes (about
// 1.8 us in pass A and 2.6 us in pass B per segment), one wave.
struct PartCand {
  long long seg_frames;
  int waves;
};
constexpr int kCands = 6;
constexpr PartCand kCandA[kCands] = {{1024, 1}, {0, 1}, {256, 1}, {4096, 1}, {1024, 2}, {4096, 2}};
constexpr PartCand kCandB[kCands] = {{2048, 1}, {0, 1}, {512, 1}, {8192, 1}, {2048, 2}, {8192, 2}};

// CTAs of the streaming passes per resident CTA slot.
#ifndef FFCA_GRID_WAVES
#define FFCA_GRID_WAVES 1
#endif

// Text of the last failed CUDA call in this thread (for ffca_last_error).
thread_local char g_last_error[256] = "";

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  return false;
}
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Plan {
  Partition pA, pB, pW;
  size_t off_info, off_ustart, off_msum;  // batch: problem tables, per-mixture sums
  size_t off_ustartW, off_bstartW;        // batch: the Wiener pass's unit starts and block ranges
  size_t off_bstartA[kCands], off_slotsA[kCands], off_bstartB[kCands], off_slotsB[kCands];  // batch candidates
  size_t off_partAdj, off_lossf, off_loss;  // adjoint: slots, per-frequency and total loss
  size_t off_cntA, off_cntB, off_logdet, off_llf, off_trace, off_pinvH, off_partA, off_partB, off_tabA, off_tabB, off_lamnext;
  size_t off_partE;  // the normal EM's pass-A slots (pass A's partition, em_nv sums each)
  size_t off_maskR;  // the masked covariances of ffca_mask_init [problems][J][I][I] complex
  size_t off_resHist;  // the resident kernel's per-iteration L2 [kResChunk][problems]
  size_t bytes;
};

ffca_status check_shape(const ffca_desc* d) {
  if (!d) return FFCA_ERR_ARG;
  if (d->prec != FFCA_PREC_FP64 && d->prec != FFCA_PREC_MIXED) return FFCA_ERR_ARG;
  if (d->F < 0 || d->N < 1 || d->ld < d->N || (d->ld % 4) != 0 || d->K < 1) return FFCA_ERR_ARG;
  if (d->I < 1 || d->J < 1) return FFCA_ERR_ARG;
  if ((d->I > 4 && d->I != 8) || d->J > 6) return FFCA_ERR_UNSUPPORTED;
  return FFCA_OK;
}

ffca_status check_pointers(const ffca_desc* d) {
  if (d->F == 0) return FFCA_OK;
  auto al = [](const void* p, uintptr_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) == 0; };
  if (!al(d->y, 16) || !al(d->v, 16) || !al(d->lambda, 8) || !al(d->P, 16)) return FFCA_ERR_ARG;
  if (!al(d->workspace, kAlign)) return FFCA_ERR_ARG;
  return FFCA_OK;
}

struct Occupancy {
  int nsm, occA, occB, occW;
};

// Resident CTAs per SM of the kernels (and the dynamic shared memory they
// need set on them).
ffca_status query_occupancy(const FastKernels* k, Occupancy* o) {
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return FFCA_ERR_CUDA;
  if (!cuda_ok(cudaDeviceGetAttribute(&o->nsm, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute"))
    return FFCA_ERR_CUDA;
  // the streaming passes take more than the default 48 KB of dynamic shared memory
  for (const void* fn : {k->estep_update, k->estep_eval})
    if (!cuda_ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->stream_smem),
                 "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)"))
      return FFCA_ERR_CUDA;
  if (!cuda_ok(cudaFuncSetAttribute(k->wcov, cudaFuncAttributeMaxDynamicSharedMemorySize, k->wcov_smem),
               "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, pass B)"))
    return FFCA_ERR_CUDA;
  if (k->estep_em &&
      (!cuda_ok(cudaFuncSetAttribute(k->estep_em, cudaFuncAttributeMaxDynamicSharedMemorySize, k->em_smem),
                "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, EM pass)") ||
       !cuda_ok(cudaFuncSetAttribute(k->psolve_em, cudaFuncAttributeMaxDynamicSharedMemorySize, k->em_solve_smem),
                "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, EM step)")))
    return FFCA_ERR_CUDA;
  if (k->pnewton && k->newton_smem > 0 &&
      !cuda_ok(cudaFuncSetAttribute(k->pnewton, cudaFuncAttributeMaxDynamicSharedMemorySize, k->newton_smem),
               "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, Newton step)"))
    return FFCA_ERR_CUDA;
  if (k->solve_smem > 0)
    for (const void* fn : {k->psolve, k->prep})
      if (!cuda_ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->solve_smem),
                   "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, solve)"))
        return FFCA_ERR_CUDA;
  o->occA = o->occB = o->occW = 0;
  const int sthreads = kGroupThreads * k->stream_groups;
  if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->occA, k->estep_update, sthreads, k->stream_smem),
               "occupancy(pass A)") ||
      !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->occB, k->wcov, kGroupThreads * k->wcov_groups,
                                                             k->wcov_smem),
               "occupancy(pass B)") ||
      !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->occW, k->wiener, kBlock, 0), "occupancy(Wiener)"))
    return FFCA_ERR_CUDA;
  if (o->occA < 1 || o->occB < 1 || o->occW < 1) {
    cudaFuncAttributes fa;
    std::memset(&fa, 0, sizeof(fa));
    cudaFuncGetAttributes(&fa, o->occA < 1 ? k->estep_update : k->wcov);
    std::snprintf(g_last_error, sizeof(g_last_error),
                  "no resident CTA: occupancy A=%d B=%d W=%d; regs=%d maxThreads=%d static=%zu requested=%d",
                  o->occA, o->occB, o->occW, fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes,
                  k->stream_smem);
    return FFCA_ERR_INTERNAL;
  }
  return FFCA_OK;
}

// Workspace layout for P problems (partitions already made).
void layout(Plan* p, const FastKernels* k, int P, int I, int J) {
  size_t off = kAlign;  // status words, global counters, inversion count
  p->off_cntA = off; off = align_up(off + sizeof(unsigned) * P);
  p->off_cntB = off; off = align_up(off + sizeof(unsigned) * P);
  p->off_logdet = off; off = align_up(off + sizeof(double) * P);
  p->off_llf = off; off = align_up(off + sizeof(double) * P);
  p->off_trace = off; off = align_up(off + sizeof(double) * kTraceCap);
  p->off_pinvH = off; off = align_up(off + sizeof(double) * 2 * I * I * (size_t)P);
  p->off_partA = off; off = align_up(off + sizeof(double) * (size_t)P * p->pA.max_slots * (J * I + 2));
  p->off_partB = off; off = align_up(off + sizeof(double) * (size_t)P * p->pB.max_slots * I * I * I);
  p->off_tabA = off; off = align_up(off + (size_t)P * k->params_a_bytes);
  p->off_tabB = off; off = align_up(off + (size_t)P * k->params_b_bytes);
  p->off_lamnext = off; off = align_up(off + sizeof(double) * (size_t)P * J * I);
  p->off_partE = off; off = align_up(off + sizeof(double) * (size_t)P * p->pA.max_slots * k->em_nv);
  p->off_maskR = off; off = align_up(off + sizeof(double) * 2 * (size_t)P * J * I * I);
  p->off_resHist = off; off = align_up(off + sizeof(double) * (size_t)kResChunk * P);
  // the adjoint kernels use pass A's partition; J I + 2 I^2 + 2 sums per slot at most
  p->off_partAdj = off; off = align_up(off + sizeof(double) * (size_t)P * p->pA.max_slots * (J * I + 2 * I * I + 2));
  p->off_lossf = off; off = align_up(off + sizeof(double) * (size_t)P);
  p->off_loss = off; off = align_up(off + sizeof(double));
  p->off_info = p->off_ustart = p->off_msum = p->off_ustartW = p->off_bstartW = 0;
  for (int q = 0; q < kCands; ++q) p->off_bstartA[q] = p->off_slotsA[q] = p->off_bstartB[q] = p->off_slotsB[q] = 0;
  p->bytes = off;
}

ffca_status make_plan(const ffca_desc* d, const FastKernels* k, Plan* p) {
  Occupancy o;
  ffca_status st = query_occupancy(k, &o);
  if (st != FFCA_OK) return st;
  const int FU = d->prec == FFCA_PREC_FP64 ? 1 : 2;
  // vector units per frequency, rounded up to even so that every tile of v
  // starts on a 16-byte boundary (ld % 4 == 0 keeps this inside the row)
  const int Uf = ((d->N + FU - 1) / FU + 1) / 2 * 2;
  const int F = d->F > 0 ? d->F : 1;
  // the streaming partitions count virtual blocks: stream_groups pipelines per CTA
  p->pA = make_partition(F, Uf, o.nsm * o.occA * k->stream_groups * FFCA_GRID_WAVES, d->N);
  p->pB = make_partition(F, Uf, o.nsm * o.occB * k->wcov_groups * FFCA_GRID_WAVES, d->N);
  // the Wiener pass also covers the padding frames (it writes them as zero)
  p->pW = make_partition(F, d->ld / FU, o.nsm * o.occW, d->N);
  p->pA.F = p->pB.F = p->pW.F = d->F;
  p->pA.Fm = p->pB.Fm = p->pW.Fm = d->F;
  layout(p, k, F, d->I, d->J);
  return FFCA_OK;
}

}  // namespace

struct TimedLaunch {
  int kind;
  cudaEvent_t start, stop;
};

struct ffca_ctx {
  ffca_desc d;  // for a batch: F = problems (M F), N unused, ld = concatenated frames
  const FastKernels* kern;
  Plan plan;
  int M;        // mixtures (1 for the single-mixture API)
  int Fm;       // frequencies per mixture
  // batch: the candidate partitions of each pass (device tables attached) and the ones in use
  Partition candA[kCands], candB[kCands];
  int curA, curB;
  // CUDA graph of the iteration loop (batch API)
  int use_graph;
  int graph_iters;
  int graph_traced;  // the cached graph writes the log-likelihood trace
  cudaGraphExec_t graph;
  cudaStream_t stream;
  char* ws;
  unsigned* status;
  unsigned* gcntA;
  unsigned* gcntB;
  unsigned long long* ops;
  int err_f;
  // update of P (kPFixedPoint unless ffca_set_p_update chose a gradient method) and its step size
  int pmode;
  double mu;
  int fault;  // injected fault for tests (kFaultNone unless ffca_test_fault set one)
  int resident;      // iterate with each problem resident on chip (ffca_set_resident)
  int max_frames;    // frames of the largest problem
  size_t res_smem;   // dynamic shared memory of the resident kernel
  // profiling
  int timing;
  unsigned long long launches[FFCA_KERNEL_KINDS];
  TimedLaunch* timed;
  size_t ntimed, captimed;
};

namespace {

FastArgs base_args(const ffca_ctx* c) {
  FastArgs a;
  std::memset(&a, 0, sizeof(a));
  a.I = c->d.I;
  a.J = c->d.J;
  a.F = c->d.F;
  a.N = c->d.N;
  a.ld = c->d.ld;
  a.K = c->d.K;
  a.y = c->d.y;
  a.v = c->d.v;
  a.lam = c->d.lambda;
  a.P = c->d.P;
  a.logdet = reinterpret_cast<double*>(c->ws + c->plan.off_logdet);
  a.llf = reinterpret_cast<double*>(c->ws + c->plan.off_llf);
  a.trace = reinterpret_cast<double*>(c->ws + c->plan.off_trace);
  a.status = c->status;
  a.ops = c->ops;
  a.tabA = c->ws + c->plan.off_tabA;
  a.tabB = c->ws + c->plan.off_tabB;
  a.inv_n = 1.0 / c->d.N;
  a.pmode = c->pmode;
  a.mu = c->mu;
  a.fault = c->fault;
  return a;
}

FastArgs pass_a_args(const ffca_ctx* c, int slot) {
  FastArgs a = base_args(c);
  a.part = c->plan.pA;
  a.part_buf = reinterpret_cast<double*>(c->ws + c->plan.off_partA);
  a.cnt = reinterpret_cast<unsigned*>(c->ws + c->plan.off_cntA);
  a.gcnt = c->gcntA;
  a.trace_slot = slot;
  return a;
}

FastArgs pass_b_args(const ffca_ctx* c, int slot) {
  FastArgs a = base_args(c);
  a.part = c->plan.pB;
  a.part_buf = reinterpret_cast<double*>(c->ws + c->plan.off_partB);
  a.cnt = reinterpret_cast<unsigned*>(c->ws + c->plan.off_cntB);
  a.gcnt = c->gcntB;
  a.trace_slot = slot;
  a.prev_part = c->plan.pA;
  a.prev_buf = reinterpret_cast<double*>(c->ws + c->plan.off_partA);
  a.lam_next = reinterpret_cast<double*>(c->ws + c->plan.off_lamnext);
  // the Gauss-Jordan / LDL^H P step reads P^{-H} of the current P and leaves that of the new one
  a.pinvH = reinterpret_cast<double*>(c->ws + c->plan.off_pinvH);
  return a;
}

// NVTX range names of the kernel kinds (FFCA_KERNEL_*): a profiler that
// records NVTX (nsys) shows every launch under its kind; without one the
// push and pop cost a branch.
const char* const kKindNames[FFCA_KERNEL_KINDS] = {
    "ffca prep", "ffca pass A", "ffca loglik", "ffca pass B", "ffca wiener",
    "ffca P step", "ffca pass A finalise", "ffca adjoint", "ffca adjoint finalise", "ffca resident"};

template <typename Args>
ffca_status launch(ffca_ctx* c, int kind, const void* fn, int grid, int block, Args& a, size_t smem = 0) {
  struct Range {  // one NVTX range around the enqueue
    explicit Range(const char* n) { nvtxRangePushA(n); }
    ~Range() { nvtxRangePop(); }
  } range(kKindNames[kind]);
  void* args[] = {&a};
  TimedLaunch* t = nullptr;
  if (c->timing && !c->use_graph) {
    if (c->ntimed == c->captimed) {
      size_t cap = c->captimed ? 2 * c->captimed : 256;
      void* p = std::realloc(c->timed, cap * sizeof(TimedLaunch));
      if (!p) return FFCA_ERR_INTERNAL;
      c->timed = static_cast<TimedLaunch*>(p);
      c->captimed = cap;
    }
    t = &c->timed[c->ntimed];
    t->kind = kind;
    if (cudaEventCreate(&t->start) != cudaSuccess) return FFCA_ERR_CUDA;
    if (cudaEventCreate(&t->stop) != cudaSuccess) {
      cudaEventDestroy(t->start);
      return FFCA_ERR_CUDA;
    }
    ++c->ntimed;
    if (cudaEventRecord(t->start, c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  }
  if (!cuda_ok(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, c->stream), "cudaLaunchKernel"))
    return FFCA_ERR_CUDA;
  ++c->launches[kind];
  if (t && cudaEventRecord(t->stop, c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  return FFCA_OK;
}

bool prep_wide(const ffca_ctx* c);

ffca_status launch_prep(ffca_ctx* c, bool want_pinv) {
  FastArgs a = base_args(c);
  // always where the P step starts from P^{-H}
  a.pinvH = (want_pinv || c->kern->pinv_step) ? reinterpret_cast<double*>(c->ws + c->plan.off_pinvH) : nullptr;
  if (prep_wide(c)) return launch(c, FFCA_KERNEL_PREP, c->kern->prep_wide, c->d.F, 32, a, 0);
  const int G = 32 / c->d.I;  // frequencies per warp
  return launch(c, FFCA_KERNEL_PREP, c->kern->prep, (c->d.F + G - 1) / G, 32, a, c->kern->solve_smem);
}

// The fixed-point step with one warp per problem (k_psolve_wide) up to this
// many problems.  Its FP64 instructions per problem are 1.5x (I = 8) to 6x
// (I = 3) those of the packed form (32 / I problems per warp), whose few
// warps leave most FP64 units idle while the problems are few.  Measured
// (mixed precision, N = 64): the packed step takes 13 - 14.5 us at I = 3,
// 18.3 - 18.7 us at I = 4 and 55 - 62 us at I = 8 from about a thousand to
// 2048 problems; the wide one 12.1 / 14.5 us at 513 / 928 problems (I = 3),
// 14.5 / 18.5 us at 513 / 1024 (I = 4) and 31 / 41 / 58 us at 513 / 1024 /
// 1664 (I = 8).  They cross near 780, 1020 and 1580 problems.
constexpr int kWideMaxProblems3 = 768;
constexpr int kWideMaxProblems4 = 1024;
constexpr int kWideMaxProblems8 = 1536;

int wide_max_problems(int I) {
  return I == 8 ? kWideMaxProblems8 : (I == 4 ? kWideMaxProblems4 : kWideMaxProblems3);
}

bool p_step_wide(const ffca_ctx* c) {
  return c->pmode == kPFixedPoint && c->kern->psolve_wide != nullptr && c->d.F <= wide_max_problems(c->d.I);
}

// The EM step and prep with one warp per problem (k_psolve_em_wide,
// k_prep_wide), on the same problem counts.
bool em_step_wide(const ffca_ctx* c) {
  return c->kern->psolve_em_wide != nullptr && c->d.F <= wide_max_problems(c->d.I);
}
bool prep_wide(const ffca_ctx* c) {
  return c->kern->prep_wide != nullptr && c->d.F <= wide_max_problems(c->d.I);
}

// Blocks of the P step: one warp per 32 / I problems (Newton and the wide
// fixed point: one block per problem), plus the trace's block.
int p_step_grid(const ffca_ctx* c, const FastArgs& b) {
  const int G = (c->pmode == kPNewton || p_step_wide(c)) ? 1 : 32 / c->d.I;
  return (c->d.F + G - 1) / G + (b.trace ? 1 : 0);
}

// Threads and dynamic shared memory of the P step's blocks.
int p_step_threads(const ffca_ctx* c) { return c->pmode == kPNewton ? c->kern->newton_threads : 32; }
size_t p_step_smem(const ffca_ctx* c) {
  if (p_step_wide(c)) return 0;  // static shared memory only
  return c->pmode == kPNewton ? c->kern->newton_smem : c->kern->solve_smem;
}

// The P step of the context's update of P (after pass B).
const void* p_step_kernel(const ffca_ctx* c) {
  if (c->pmode == kPNewton) return c->kern->pnewton;
  if (p_step_wide(c)) return c->kern->psolve_wide;
  return c->pmode == kPGradient || c->pmode == kPNatural ? c->kern->pgrad : c->kern->psolve;
}

int finals_grid(const ffca_ctx* c) { return (c->d.F + kFinalWarps - 1) / kFinalWarps; }

// Iterations with each problem resident on chip: chunks of up to kResChunk
// iterations per launch; with a trace each chunk's per-problem L2 are summed
// into trace slots 0 .. n-1 and copied to host[t0 ..] (synchronising).
bool resident_active(const ffca_ctx* c) { return c->resident && c->pmode == kPFixedPoint; }

ffca_status enqueue_resident(ffca_ctx* c, int iters, double* host_trace) {
  ResArgs r;
  std::memset(&r, 0, sizeof(r));
  r.a = base_args(c);
  r.a.part = c->plan.pA;
  r.a.pinvH = reinterpret_cast<double*>(c->ws + c->plan.off_pinvH);
  r.hist = reinterpret_cast<double*>(c->ws + c->plan.off_resHist);
  double* dtrace = reinterpret_cast<double*>(c->ws + c->plan.off_trace);
  for (int t0 = 0; t0 < iters; t0 += kResChunk) {
    r.iters = std::min(kResChunk, iters - t0);
    ffca_status st = launch(c, FFCA_KERNEL_RESIDENT, c->kern->resident, c->d.F, kResThreads, r, c->res_smem);
    if (st != FFCA_OK) return st;
    if (host_trace) {
      k_res_trace<<<r.iters, 32, 0, c->stream>>>(r.hist, c->d.F, dtrace, 0);
      if (!cuda_ok(cudaGetLastError(), "k_res_trace") ||
          !cuda_ok(cudaMemcpyAsync(host_trace + t0, dtrace, sizeof(double) * r.iters, cudaMemcpyDeviceToHost,
                                   c->stream), "cudaMemcpyAsync(trace)") ||
          !cuda_ok(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize"))
        return FFCA_ERR_CUDA;
    }
  }
  return FFCA_OK;
}

// One iteration with the normal EM update of P: pass A with the EM sums
// (on pass A's partition, em_groups pipeline groups per CTA) and the
// per-problem EM step; no pass B.  With `trace` the step's
// last block sums the problems' L2 of the entering state into trace slot
// `slot`.
ffca_status launch_em_iteration(ffca_ctx* c, int slot, bool trace) {
  FastArgs a = base_args(c);
  a.part = c->plan.pA;
  a.part_buf = reinterpret_cast<double*>(c->ws + c->plan.off_partE);
  a.trace_slot = slot;
  a.pinvH = reinterpret_cast<double*>(c->ws + c->plan.off_pinvH);
  a.gcnt = reinterpret_cast<unsigned*>(c->ws + 28);
  if (!trace) a.trace = nullptr;
  const int eg = c->kern->em_groups;
  ffca_status st = launch(c, FFCA_KERNEL_ESTEP, c->kern->estep_em, (a.part.nblocks + eg - 1) / eg,
                          kGroupThreads * eg, a, c->kern->em_smem);
  if (st != FFCA_OK) return st;
  if (em_step_wide(c)) return launch(c, FFCA_KERNEL_PSOLVE, c->kern->psolve_em_wide, c->d.F, 32, a, 0);
  const int G = 32 / c->d.I;
  return launch(c, FFCA_KERNEL_PSOLVE, c->kern->psolve_em, (c->d.F + G - 1) / G, 32, a, c->kern->em_solve_smem);
}

// CTAs of a streaming pass: each runs stream_groups (pass A) or wcov_groups
// (pass B) virtual blocks of the partition.
int stream_grid(const ffca_ctx* c, const Partition& p) {
  return (p.nblocks + c->kern->stream_groups - 1) / c->kern->stream_groups;
}
int stream_threads(const ffca_ctx* c) { return kGroupThreads * c->kern->stream_groups; }
int wcov_grid(const ffca_ctx* c, const Partition& p) {
  return (p.nblocks + c->kern->wcov_groups - 1) / c->kern->wcov_groups;
}
int wcov_threads(const ffca_ctx* c) { return kGroupThreads * c->kern->wcov_groups; }

void drop_timed(ffca_ctx* c) {
  for (size_t k = 0; k < c->ntimed; ++k) {
    cudaEventDestroy(c->timed[k].start);
    cudaEventDestroy(c->timed[k].stop);
  }
  c->ntimed = 0;
}

ffca_status read_status(ffca_ctx* c) {
  unsigned h[2] = {0, 0};
  if (cudaMemcpyAsync(h, c->status, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return FFCA_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  if (h[0] != 0) {
    c->err_f = (int)h[1];
    return (ffca_status)h[0];
  }
  c->err_f = -1;
  return FFCA_OK;
}

}  // namespace

namespace {

// The launches of `iters` iterations, without host copies (capturable).
// traced (not with the resident form; iters < kTraceCap): the
// log-likelihood of the state entering iteration t goes to device trace
// slot t and that of the final state to slot iters.
ffca_status enqueue_iterations(ffca_ctx* c, int iters, bool traced = false) {
  ffca_status st = launch_prep(c, resident_active(c));
  if (st != FFCA_OK) return st;
  if (resident_active(c)) return enqueue_resident(c, iters, nullptr);
  for (int t = 0; t < iters; ++t) {
    const int slot = t % kTraceCap;
    if (c->pmode == kPEM) {
      if ((st = launch_em_iteration(c, slot, traced)) != FFCA_OK) return st;
      continue;
    }
    FastArgs a = pass_a_args(c, slot);
    if ((st = launch(c, FFCA_KERNEL_ESTEP, c->kern->estep_update, stream_grid(c, a.part), stream_threads(c), a,
                     c->kern->stream_smem)) != FFCA_OK)
      return st;
    FastArgs b = pass_b_args(c, slot);
    if (!traced) b.trace = nullptr;  // no trace: no trace block in the P step
    if ((st = launch(c, FFCA_KERNEL_WCOV, c->kern->wcov, wcov_grid(c, b.part), wcov_threads(c), b,
                     c->kern->wcov_smem)) != FFCA_OK)
      return st;
    if ((st = launch(c, FFCA_KERNEL_PSOLVE, p_step_kernel(c), p_step_grid(c, b), p_step_threads(c), b, p_step_smem(c))) != FFCA_OK) return st;
  }
  if (traced) {  // the log-likelihood of the final state
    FastArgs a = pass_a_args(c, iters % kTraceCap);
    if ((st = launch(c, FFCA_KERNEL_LOGLIK, c->kern->estep_eval, stream_grid(c, a.part), stream_threads(c), a,
                     c->kern->stream_smem)) != FFCA_OK)
      return st;
    if ((st = launch(c, FFCA_KERNEL_AFINAL, c->kern->afinal_eval, finals_grid(c), 32 * kFinalWarps, a)) != FFCA_OK)
      return st;
  }
  return FFCA_OK;
}

// Iterations replayed from a CUDA graph of the whole launch sequence,
// captured on the first call for a given iteration count (and trace or
// none).  With ll_trace the graph writes the trace slots, which are then
// copied to ll_trace[0 .. iters] (synchronising, with the status).
ffca_status iterate_graph(ffca_ctx* c, int iters, double* ll_trace = nullptr) {
  const bool traced = ll_trace != nullptr;
  if (!c->graph || c->graph_iters != iters || c->graph_traced != (traced ? 1 : 0)) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    // capture on a private stream (the legacy default stream cannot be
    // captured); nothing runs during the capture, so no ordering is needed
    cudaStream_t cap = nullptr;
    if (!cuda_ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreateWithFlags"))
      return FFCA_ERR_CUDA;
    if (!cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
      cudaStreamDestroy(cap);
      return FFCA_ERR_CUDA;
    }
    const cudaStream_t user = c->stream;
    c->stream = cap;
    unsigned long long saved[FFCA_KERNEL_KINDS];
    std::memcpy(saved, c->launches, sizeof(saved));
    ffca_status st = enqueue_iterations(c, iters, traced);
    std::memcpy(c->launches, saved, sizeof(saved));  // captured, not yet run
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    c->stream = user;
    cudaStreamDestroy(cap);
    if (st != FFCA_OK || !cuda_ok(e, "cudaStreamEndCapture")) {
      if (g) cudaGraphDestroy(g);
      return st != FFCA_OK ? st : FFCA_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (!cuda_ok(ei, "cudaGraphInstantiate")) {
      c->graph = nullptr;
      return FFCA_ERR_CUDA;
    }
    c->graph_iters = iters;
    c->graph_traced = traced ? 1 : 0;
  }
  if (!cuda_ok(cudaGraphLaunch(c->graph, c->stream), "cudaGraphLaunch")) return FFCA_ERR_CUDA;
  c->launches[FFCA_KERNEL_PREP] += 1;
  if (resident_active(c)) {
    c->launches[FFCA_KERNEL_RESIDENT] += (iters + kResChunk - 1) / kResChunk;
    return FFCA_OK;
  }
  c->launches[FFCA_KERNEL_ESTEP] += iters;
  if (c->pmode != kPEM) c->launches[FFCA_KERNEL_WCOV] += iters;
  c->launches[FFCA_KERNEL_PSOLVE] += iters;
  if (!traced) return FFCA_OK;
  c->launches[FFCA_KERNEL_LOGLIK] += 1;
  c->launches[FFCA_KERNEL_AFINAL] += 1;
  const double* dtrace = reinterpret_cast<const double*>(c->ws + c->plan.off_trace);
  if (!cuda_ok(cudaMemcpyAsync(ll_trace, dtrace, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost, c->stream),
               "cudaMemcpyAsync(trace)"))
    return FFCA_ERR_CUDA;
  return read_status(c);
}

// Per-mixture sums of the per-problem log-likelihoods (block m sums the F
// problems of mixture m in a fixed order).
__global__ void k_mixture_sums(const double* llf, int F, double* out) {
  __shared__ double part[32];
  const int m = blockIdx.x;
  double s = 0.0;
  for (int f = threadIdx.x; f < F; f += blockDim.x) s += __ldcg(llf + (size_t)m * F + f);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) out[m] = t;
  }
}

// Gradients of NLL (se = false) or of the Wiener squared error (se = true)
// at the context's current state: k_prep (P^{-H}, ln|det P|^2), the
// streaming adjoint pass, the per-frequency finalisation.
ffca_status adjoint(ffca_ctx* c, bool se, const void* s, void* dv, double* dlam, double* dP, double* loss) {
  if (!c) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    if (loss) *loss = 0.0;
    return FFCA_OK;
  }
  auto al = [](const void* q, uintptr_t n) { return q && (reinterpret_cast<uintptr_t>(q) % n) == 0; };
  if (!al(dv, 16) || !al(dlam, 8) || !al(dP, 16) || (se && !al(s, 16))) return FFCA_ERR_ARG;
  const AdjKernels* k = adj_kernels(c->d.prec, c->d.I, c->d.J);
  if (!k) return FFCA_ERR_UNSUPPORTED;
  ffca_status st = launch_prep(c, true);
  if (st != FFCA_OK) return st;
  AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.part = c->plan.pA;
  a.F = c->d.F;
  a.N = c->d.N;
  a.ld = c->d.ld;
  a.y = c->d.y;
  a.v = c->d.v;
  a.lam = c->d.lambda;
  a.P = c->d.P;
  a.pinvH = reinterpret_cast<const double*>(c->ws + c->plan.off_pinvH);
  a.logdet = reinterpret_cast<const double*>(c->ws + c->plan.off_logdet);
  a.s = s;
  a.dv = dv;
  a.dlam = dlam;
  a.dP = dP;
  a.part_buf = reinterpret_cast<double*>(c->ws + c->plan.off_partAdj);
  a.lossf = reinterpret_cast<double*>(c->ws + c->plan.off_lossf);
  a.loss = reinterpret_cast<double*>(c->ws + c->plan.off_loss);
  a.gcnt = reinterpret_cast<unsigned*>(c->ws + 24);
  a.status = c->status;
  if ((st = launch(c, FFCA_KERNEL_ADJ, se ? k->se : k->nll, a.part.nblocks, kBlock, a)) != FFCA_OK) return st;
  if ((st = launch(c, FFCA_KERNEL_ADJ_FINAL, se ? k->se_final : k->nll_final, (c->d.F + 3) / 4, 128, a)) !=
      FFCA_OK)
    return st;
  if (!loss) return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
  if (!cuda_ok(cudaMemcpyAsync(loss, a.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync"))
    return FFCA_ERR_CUDA;
  return read_status(c);
}

}  // namespace

extern "C" {

size_t ffca_workspace_size(const ffca_desc* d) {
  if (check_shape(d) != FFCA_OK) return 0;
  const FastKernels* k = fast_kernels(d->prec, d->I, d->J);
  if (!k) return 0;
  Plan p;
  if (make_plan(d, k, &p) != FFCA_OK) return 0;
  return p.bytes;
}

ffca_status ffca_init(ffca_ctx** out, const ffca_desc* d) {
  if (!out) return FFCA_ERR_ARG;
  *out = nullptr;
  ffca_status st = check_shape(d);
  if (st != FFCA_OK) return st;
  if ((st = check_pointers(d)) != FFCA_OK) return st;
  const FastKernels* k = fast_kernels(d->prec, d->I, d->J);
  if (!k) return FFCA_ERR_UNSUPPORTED;
  Plan p;
  if ((st = make_plan(d, k, &p)) != FFCA_OK) return st;
  if (d->F > 0 && d->workspace_bytes < p.bytes) return FFCA_ERR_ARG;
  ffca_ctx* c = static_cast<ffca_ctx*>(std::calloc(1, sizeof(ffca_ctx)));
  if (!c) return FFCA_ERR_INTERNAL;
  c->d = *d;
  c->kern = k;
  c->plan = p;
  c->stream = static_cast<cudaStream_t>(d->stream);
  c->ws = static_cast<char*>(d->workspace);
  c->status = reinterpret_cast<unsigned*>(c->ws);
  c->gcntA = reinterpret_cast<unsigned*>(c->ws + 16);
  c->gcntB = reinterpret_cast<unsigned*>(c->ws + 20);
  c->ops = reinterpret_cast<unsigned long long*>(c->ws + 32);
  c->err_f = -1;
  c->M = 1;
  c->Fm = d->F;
  c->max_frames = d->N;
  if (d->F > 0 && cudaMemsetAsync(c->ws, 0, p.bytes, c->stream) != cudaSuccess) {
    std::free(c);
    return FFCA_ERR_CUDA;
  }
  *out = c;
  return FFCA_OK;
}

ffca_status ffca_iterate(ffca_ctx* c, int iters, double* ll_trace) {
  if (!c || iters < 0) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    if (ll_trace)
      for (int t = 0; t <= iters; ++t) ll_trace[t] = 0.0;
    return FFCA_OK;
  }
  if (c->use_graph && (!ll_trace || (iters < kTraceCap && !resident_active(c))))
    return iterate_graph(c, iters, ll_trace);
  if (resident_active(c)) {
    ffca_status st = launch_prep(c, true);
    if (st == FFCA_OK) st = enqueue_resident(c, iters, ll_trace);
    if (st != FFCA_OK) return st;
    if (!ll_trace) return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
    // L2 of the final state
    FastArgs a = pass_a_args(c, 0);
    if ((st = launch(c, FFCA_KERNEL_LOGLIK, c->kern->estep_eval, stream_grid(c, a.part), stream_threads(c), a,
                     c->kern->stream_smem)) != FFCA_OK ||
        (st = launch(c, FFCA_KERNEL_AFINAL, c->kern->afinal_eval, finals_grid(c), 32 * kFinalWarps, a)) != FFCA_OK)
      return st;
    if (!cuda_ok(cudaMemcpyAsync(ll_trace + iters, a.trace, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                 "cudaMemcpyAsync(trace)"))
      return FFCA_ERR_CUDA;
    return read_status(c);
  }
  ffca_status st = launch_prep(c, false);
  if (st != FFCA_OK) return st;
  const double* dtrace = reinterpret_cast<const double*>(c->ws + c->plan.off_trace);
  int flushed = 0;  // first trace index not yet copied to the host
  for (int t = 0; t <= iters; ++t) {
    const int slot = t % kTraceCap;
    if (t < iters && c->pmode == kPEM) {
      if ((st = launch_em_iteration(c, slot, ll_trace != nullptr)) != FFCA_OK) return st;
    } else if (t < iters) {
      FastArgs a = pass_a_args(c, slot);
      if ((st = launch(c, FFCA_KERNEL_ESTEP, c->kern->estep_update, stream_grid(c, a.part), stream_threads(c), a,
                      c->kern->stream_smem)) != FFCA_OK)
        return st;
      FastArgs b = pass_b_args(c, slot);
      if (!ll_trace) b.trace = nullptr;  // no trace block in the P step
      if ((st = launch(c, FFCA_KERNEL_WCOV, c->kern->wcov, wcov_grid(c, b.part), wcov_threads(c), b,
                      c->kern->wcov_smem)) != FFCA_OK)
        return st;
      if ((st = launch(c, FFCA_KERNEL_PSOLVE, p_step_kernel(c), p_step_grid(c, b), p_step_threads(c), b, p_step_smem(c))) != FFCA_OK)
        return st;
    } else if (ll_trace) {
      FastArgs a = pass_a_args(c, slot);
      if ((st = launch(c, FFCA_KERNEL_LOGLIK, c->kern->estep_eval, stream_grid(c, a.part), stream_threads(c), a,
                      c->kern->stream_smem)) != FFCA_OK)
        return st;
      if ((st = launch(c, FFCA_KERNEL_AFINAL, c->kern->afinal_eval, finals_grid(c), 32 * kFinalWarps, a)) !=
          FFCA_OK)
        return st;
    }
    if (ll_trace && (slot == kTraceCap - 1 || t == iters)) {
      const int n = t - flushed + 1;
      if (cudaMemcpyAsync(ll_trace + flushed, dtrace, sizeof(double) * n, cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess)
        return FFCA_ERR_CUDA;
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
      flushed = t + 1;
    }
  }
  if (ll_trace) return read_status(c);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

ffca_status ffca_loglik(ffca_ctx* c, double* ll) {
  if (!c || !ll) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    *ll = 0.0;
    return FFCA_OK;
  }
  ffca_status st = launch_prep(c, false);
  if (st != FFCA_OK) return st;
  FastArgs a = pass_a_args(c, 0);
  if ((st = launch(c, FFCA_KERNEL_LOGLIK, c->kern->estep_eval, stream_grid(c, a.part), stream_threads(c), a,
                      c->kern->stream_smem)) != FFCA_OK)
    return st;
  if ((st = launch(c, FFCA_KERNEL_AFINAL, c->kern->afinal_eval, finals_grid(c), 32 * kFinalWarps, a)) != FFCA_OK)
    return st;
  if (cudaMemcpyAsync(ll, a.trace, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return FFCA_ERR_CUDA;
  return read_status(c);
}

ffca_status ffca_wiener(ffca_ctx* c, void* out) {
  if (!c) return FFCA_ERR_ARG;
  if (c->d.F == 0) return FFCA_OK;
  if (!out || (reinterpret_cast<uintptr_t>(out) % 16) != 0) return FFCA_ERR_ARG;
  ffca_status st = launch_prep(c, true);
  if (st != FFCA_OK) return st;
  FastArgs a = base_args(c);
  a.part = c->plan.pW;
  a.pinvH = reinterpret_cast<double*>(c->ws + c->plan.off_pinvH);
  a.out = out;
  return launch(c, FFCA_KERNEL_WIENER, c->kern->wiener, a.part.nblocks, kBlock, a);
}

ffca_status ffca_wiener_host(ffca_ctx* c, void* out_dev, void* out_host) {
  if (!c || !out_host) return FFCA_ERR_ARG;
  ffca_status st = ffca_wiener(c, out_dev);
  if (st != FFCA_OK) return st;
  const size_t rsz = c->d.prec == FFCA_PREC_FP64 ? 8 : 4;
  // J I frequencies-per-mixture rows of ld frames (a batch: the mixtures' blocks, ld in total)
  const size_t bytes = (size_t)c->d.J * c->d.I * c->Fm * c->d.ld * 2 * rsz;
  if (bytes && cudaMemcpyAsync(out_host, out_dev, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return FFCA_ERR_CUDA;
  return read_status(c);
}

ffca_status ffca_nll_grad(ffca_ctx* c, void* dv, double* dlam, double* dP, double* loss) {
  return adjoint(c, false, nullptr, dv, dlam, dP, loss);
}

ffca_status ffca_wiener_se_grad(ffca_ctx* c, const void* s, void* dv, double* dlam, double* dP, double* loss) {
  return adjoint(c, true, s, dv, dlam, dP, loss);
}

ffca_status ffca_timing_enable(ffca_ctx* c, int enable) {
  if (!c) return FFCA_ERR_ARG;
  c->timing = enable ? 1 : 0;
  return FFCA_OK;
}

ffca_status ffca_timing_read(ffca_ctx* c, double* ms, unsigned long long* launches) {
  if (!c) return FFCA_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FFCA_ERR_CUDA;
  double tot[FFCA_KERNEL_KINDS] = {};
  ffca_status st = FFCA_OK;
  for (size_t k = 0; k < c->ntimed; ++k) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, c->timed[k].start, c->timed[k].stop) != cudaSuccess) st = FFCA_ERR_CUDA;
    tot[c->timed[k].kind] += e;
  }
  drop_timed(c);
  for (int k = 0; k < FFCA_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = tot[k];
    if (launches) launches[k] = c->launches[k];
    c->launches[k] = 0;
  }
  return st;
}

ffca_status ffca_sync(ffca_ctx* c) {
  if (!c) return FFCA_ERR_ARG;
  if (c->d.F == 0) return cudaStreamSynchronize(c->stream) == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
  return read_status(c);
}

int ffca_error_frequency(const ffca_ctx* c) { return c ? c->err_f : -1; }

ffca_status ffca_inversion_count(ffca_ctx* c, unsigned long long* count) {
  if (!c || !count) return FFCA_ERR_ARG;
  if (c->d.F == 0) {
    *count = 0;
    return FFCA_OK;
  }
  if (cudaMemcpyAsync(count, c->ops, sizeof(*count), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return FFCA_ERR_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

ffca_status ffca_upload(ffca_ctx* c, const void* y_host, const void* v_host, const double* lam_host,
                        const double* P_host) {
  if (!c) return FFCA_ERR_ARG;
  const ffca_desc& d = c->d;
  const size_t rsz = d.prec == FFCA_PREC_FP64 ? 8 : 4;
  const size_t ybytes = (size_t)d.I * c->Fm * d.ld * 2 * rsz;
  const size_t vbytes = (size_t)d.J * c->Fm * d.ld * rsz;
  const size_t lbytes = (size_t)d.F * d.J * d.I * sizeof(double);
  const size_t pbytes = (size_t)d.F * d.I * d.I * 2 * sizeof(double);
  auto cp = [&](void* dst, const void* src, size_t n) {
    return (src == nullptr || n == 0 ||
            cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream) == cudaSuccess);
  };
  if (!cp(const_cast<void*>(d.y), y_host, ybytes) || !cp(d.v, v_host, vbytes) ||
      !cp(d.lambda, lam_host, lbytes) || !cp(d.P, P_host, pbytes))
    return FFCA_ERR_CUDA;
  return FFCA_OK;
}

ffca_status ffca_download(ffca_ctx* c, void* v_host, double* lam_host, double* P_host) {
  if (!c) return FFCA_ERR_ARG;
  const ffca_desc& d = c->d;
  const size_t rsz = d.prec == FFCA_PREC_FP64 ? 8 : 4;
  const size_t vbytes = (size_t)d.J * c->Fm * d.ld * rsz;
  const size_t lbytes = (size_t)d.F * d.J * d.I * sizeof(double);
  const size_t pbytes = (size_t)d.F * d.I * d.I * 2 * sizeof(double);
  auto cp = [&](void* dst, const void* src, size_t n) {
    return (dst == nullptr || n == 0 ||
            cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream) == cudaSuccess);
  };
  if (!cp(v_host, d.v, vbytes) || !cp(lam_host, d.lambda, lbytes) || !cp(P_host, d.P, pbytes))
    return FFCA_ERR_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

void ffca_destroy(ffca_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  drop_timed(c);
  std::free(c->timed);
  std::free(c);
}

const char* ffca_last_error(void) { return g_last_error; }

const char* ffca_status_str(ffca_status s) {
  switch (s) {
    case FFCA_OK: return "ok";
    case FFCA_ERR_ARG: return "invalid argument";
    case FFCA_ERR_CUDA: return "CUDA error";
    case FFCA_ERR_NONFINITE: return "non-finite or non-positive value";
    case FFCA_ERR_SINGULAR: return "singular per-frequency system";
    case FFCA_ERR_TIMEOUT: return "device wait timed out";
    case FFCA_ERR_INTERNAL: return "internal error";
    case FFCA_ERR_UNSUPPORTED: return "unsupported (I, J)";
  }
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Iteration without any allocation.
//
// Some callers cannot allocate device memory at the point where they run the
// estimation: a real-time audio thread (hearing aid, online enhancement) must
// not call cudaMalloc, which can block and synchronise the device; a plugin
// inside a host application may have no allocator of its own; a system with a
// fixed, pre-planned memory map may forbid late allocations.  For them,
// ffca_iterate_noalloc takes its scratch (partial sums, arrival counters,
// status word, trace) from the array below, which is part of the library
// image: every GPU that loads the library holds it until the process exits.
namespace {

constexpr size_t kNoallocScratchBytes = FFCA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol itself is only a host-side stand-in, never a device address.
std::atomic<void*> g_noalloc_addr[kMaxDevices];

ffca_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FFCA_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FFCA_ERR_UNSUPPORTED;
  void* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FFCA_ERR_CUDA;
    g_noalloc_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return FFCA_OK;
}

}  // namespace

extern "C" ffca_status ffca_iterate_noalloc(const ffca_desc* d, int iters, double* ll_trace) {
  if (iters < 0) return FFCA_ERR_ARG;
  ffca_status st = check_shape(d);
  if (st != FFCA_OK) return st;
  const FastKernels* k = fast_kernels(d->prec, d->I, d->J);
  if (!k) return FFCA_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  if ((st = noalloc_scratch(&scratch)) != FFCA_OK) return st;
  ffca_desc dd = *d;
  dd.workspace = scratch;
  dd.workspace_bytes = kNoallocScratchBytes;
  if ((st = check_pointers(&dd)) != FFCA_OK) return st;
  Plan p;
  if ((st = make_plan(&dd, k, &p)) != FFCA_OK) return st;
  if (p.bytes > kNoallocScratchBytes) return FFCA_ERR_ARG;  // problem too large for the fixed scratch
  // The context lives on this call's stack; nothing is allocated.
  ffca_ctx c;
  std::memset(&c, 0, sizeof(c));
  c.d = dd;
  c.kern = k;
  c.plan = p;
  c.stream = static_cast<cudaStream_t>(dd.stream);
  c.ws = static_cast<char*>(scratch);
  c.status = reinterpret_cast<unsigned*>(c.ws);
  c.gcntA = reinterpret_cast<unsigned*>(c.ws + 16);
  c.gcntB = reinterpret_cast<unsigned*>(c.ws + 20);
  c.ops = reinterpret_cast<unsigned long long*>(c.ws + 32);
  c.err_f = -1;
  c.M = 1;  // as ffca_init: one mixture of F frequencies
  c.Fm = dd.F;
  if (dd.F == 0) {
    if (ll_trace)
      for (int t = 0; t <= iters; ++t) ll_trace[t] = 0.0;
    return FFCA_OK;
  }
  // The previous call left its partials, counters and status in the shared
  // scratch: the counters and the status word must start at zero.
  // Every return after the first enqueue waits for the stream first, so that
  // no kernel of this call still uses the shared scratch when the next call
  // clears it (the wait's own result is not the call's error).
  if (cudaMemsetAsync(c.ws, 0, p.bytes, c.stream) != cudaSuccess) {
    cudaStreamSynchronize(c.stream);
    return FFCA_ERR_CUDA;
  }
  st = ffca_iterate(&c, iters, ll_trace);
  if (st != FFCA_OK) {
    cudaStreamSynchronize(c.stream);
    return st;
  }
  return read_status(&c);
}

// ---------------------------------------------------------------------------
// Batches of mixtures of uneven length: every (mixture, frequency) pair is
// one problem of the ragged partition; the same kernels run all of them.
namespace {

ffca_status batch_check(const ffca_batch_desc* d) {
  if (!d || !d->frame_offset || !d->N) return FFCA_ERR_ARG;
  if (d->prec != FFCA_PREC_FP64 && d->prec != FFCA_PREC_MIXED) return FFCA_ERR_ARG;
  if (d->M < 1 || d->F < 1 || d->K < 1 || d->I < 1 || d->J < 1) return FFCA_ERR_ARG;
  if ((d->I > 4 && d->I != 8) || d->J > 6) return FFCA_ERR_UNSUPPORTED;
  if (d->frame_offset[0] != 0 || d->ld != d->frame_offset[d->M] || d->ld > (1ll << 30)) return FFCA_ERR_ARG;
  if ((long long)d->M * d->F > (1ll << 30)) return FFCA_ERR_ARG;
  for (int m = 0; m < d->M; ++m) {
    const long long o0 = d->frame_offset[m], o1 = d->frame_offset[m + 1];
    if (o0 % 4 != 0 || o1 % 4 != 0 || d->N[m] < 1 || (o1 - o0) < d->N[m]) return FFCA_ERR_ARG;
  }
  return FFCA_OK;
}

// Host copies of a batch's device tables.
struct BatchTables {
  std::vector<ProbInfo> info;
  std::vector<long long> ustart;
  std::vector<long long> ustartW, bstartW;  // the Wiener pass: every frame of each row, padding included
  std::vector<int2> slotsW;
  Partition candW;
  std::vector<long long> bstartA[kCands], bstartB[kCands];
  std::vector<int2> slotsA[kCands], slotsB[kCands];
  Partition candA[kCands], candB[kCands];
};

ffca_status batch_plan(const ffca_batch_desc* d, const FastKernels* k, Plan* p, BatchTables* t) {
  Occupancy o;
  ffca_status st = query_occupancy(k, &o);
  if (st != FFCA_OK) return st;
  const int FU = d->prec == FFCA_PREC_FP64 ? 1 : 2;
  const int P = d->M * d->F;
  t->info.resize(P);
  t->ustart.resize(P + 1);
  long long u = 0;
  for (int m = 0; m < d->M; ++m) {
    const int Uf = ((d->N[m] + FU - 1) / FU + 1) / 2 * 2;  // even, inside the mixture's padded frames
    for (int f = 0; f < d->F; ++f) {
      const int q = m * d->F + f;
      t->info[q] = ProbInfo{d->frame_offset[m], f, d->N[m], 1.0 / d->N[m],
                            (int)(d->frame_offset[m + 1] - d->frame_offset[m])};
      t->ustart[q] = u;
      u += Uf;
    }
  }
  t->ustart[P] = u;
  // the Wiener pass covers the padding frames of each row too (it writes them as zero)
  t->ustartW.resize(P + 1);
  long long uw = 0;
  for (int m = 0; m < d->M; ++m)
    for (int f = 0; f < d->F; ++f) {
      t->ustartW[m * d->F + f] = uw;
      uw += (d->frame_offset[m + 1] - d->frame_offset[m]) / FU;
    }
  t->ustartW[P] = uw;
  t->bstartW.resize(o.nsm * o.occW + 1);
  t->slotsW.resize(P);
  t->candW = make_partition_ragged(P, d->F, t->ustartW.data(), o.nsm * o.occW, 0, t->bstartW.data(),
                                   t->slotsW.data());
  t->bstartW.resize(t->candW.nblocks + 1);
  const int slotsA = o.nsm * o.occA * k->stream_groups, slotsB = o.nsm * o.occB * k->wcov_groups;
  int msA = 1, msB = 1;
  for (int c = 0; c < kCands; ++c) {
    const int maxA = slotsA * kCandA[c].waves, maxB = slotsB * kCandB[c].waves;
    t->bstartA[c].resize(maxA + 1);
    t->bstartB[c].resize(maxB + 1);
    t->slotsA[c].resize(P);
    t->slotsB[c].resize(P);
    t->candA[c] = make_partition_ragged(P, d->F, t->ustart.data(), maxA, kCandA[c].seg_frames / FU,
                                        t->bstartA[c].data(), t->slotsA[c].data());
    t->candB[c] = make_partition_ragged(P, d->F, t->ustart.data(), maxB, kCandB[c].seg_frames / FU,
                                        t->bstartB[c].data(), t->slotsB[c].data());
    t->bstartA[c].resize(t->candA[c].nblocks + 1);
    t->bstartB[c].resize(t->candB[c].nblocks + 1);
    msA = std::max(msA, t->candA[c].max_slots);
    msB = std::max(msB, t->candB[c].max_slots);
  }
  // one slot stride for every candidate: the buffers hold the largest
  for (int c = 0; c < kCands; ++c) {
    t->candA[c].max_slots = msA;
    t->candB[c].max_slots = msB;
  }
  p->pA = t->candA[0];
  p->pB = t->candB[0];
  p->pW = t->candW;
  layout(p, k, P, d->I, d->J);
  size_t off = p->bytes;
  p->off_info = off; off = align_up(off + sizeof(ProbInfo) * (size_t)P);
  p->off_ustart = off; off = align_up(off + sizeof(long long) * (size_t)(P + 1));
  p->off_ustartW = off; off = align_up(off + sizeof(long long) * (size_t)(P + 1));
  p->off_bstartW = off; off = align_up(off + sizeof(long long) * t->bstartW.size());
  p->off_msum = off; off = align_up(off + sizeof(double) * (size_t)d->M);
  for (int c = 0; c < kCands; ++c) {
    p->off_bstartA[c] = off; off = align_up(off + sizeof(long long) * t->bstartA[c].size());
    p->off_bstartB[c] = off; off = align_up(off + sizeof(long long) * t->bstartB[c].size());
    p->off_slotsA[c] = off; off = align_up(off + sizeof(int2) * (size_t)P);
    p->off_slotsB[c] = off; off = align_up(off + sizeof(int2) * (size_t)P);
  }
  p->bytes = off;
  return FFCA_OK;
}

// Switch a batch context to candidates (ia, ib); a captured graph holds the
// old partitions and is dropped.
void use_candidates(ffca_ctx* c, int ia, int ib) {
  c->curA = ia;
  c->curB = ib;
  c->plan.pA = c->candA[ia];
  c->plan.pB = c->candB[ib];
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

}  // namespace

extern "C" {

size_t ffca_batch_workspace_size(const ffca_batch_desc* d) {
  if (batch_check(d) != FFCA_OK) return 0;
  const FastKernels* k = fast_kernels(d->prec, d->I, d->J);
  if (!k) return 0;
  Plan p;
  BatchTables t;
  if (batch_plan(d, k, &p, &t) != FFCA_OK) return 0;
  return p.bytes;
}

ffca_status ffca_batch_init(ffca_batch_ctx** out, const ffca_batch_desc* d) {
  if (!out) return FFCA_ERR_ARG;
  *out = nullptr;
  ffca_status st = batch_check(d);
  if (st != FFCA_OK) return st;
  auto al = [](const void* q, uintptr_t a) { return q && (reinterpret_cast<uintptr_t>(q) % a) == 0; };
  if (!al(d->y, 16) || !al(d->v, 16) || !al(d->lambda, 8) || !al(d->P, 16) || !al(d->workspace, kAlign))
    return FFCA_ERR_ARG;
  const FastKernels* k = fast_kernels(d->prec, d->I, d->J);
  if (!k) return FFCA_ERR_UNSUPPORTED;
  Plan p;
  BatchTables t;
  if ((st = batch_plan(d, k, &p, &t)) != FFCA_OK) return st;
  if (d->workspace_bytes < p.bytes) return FFCA_ERR_ARG;
  ffca_ctx* c = static_cast<ffca_ctx*>(std::calloc(1, sizeof(ffca_ctx)));
  if (!c) return FFCA_ERR_INTERNAL;
  c->d.I = d->I;
  c->d.J = d->J;
  c->d.F = d->M * d->F;  // problems
  c->d.N = 1;            // per-problem frame counts live in the tables
  c->d.ld = (int)d->ld;
  c->d.K = d->K;
  c->d.prec = d->prec;
  c->d.y = d->y;
  c->d.v = d->v;
  c->d.lambda = d->lambda;
  c->d.P = d->P;
  c->d.workspace = d->workspace;
  c->d.workspace_bytes = d->workspace_bytes;
  c->d.stream = d->stream;
  c->kern = k;
  c->plan = p;
  c->M = d->M;
  c->Fm = d->F;
  c->max_frames = *std::max_element(d->N, d->N + d->M);
  c->stream = static_cast<cudaStream_t>(d->stream);
  c->ws = static_cast<char*>(d->workspace);
  c->status = reinterpret_cast<unsigned*>(c->ws);
  c->gcntA = reinterpret_cast<unsigned*>(c->ws + 16);
  c->gcntB = reinterpret_cast<unsigned*>(c->ws + 20);
  c->ops = reinterpret_cast<unsigned long long*>(c->ws + 32);
  c->err_f = -1;
  const ProbInfo* dinfo = reinterpret_cast<const ProbInfo*>(c->ws + p.off_info);
  const long long* dustart = reinterpret_cast<const long long*>(c->ws + p.off_ustart);
  auto up = [&](size_t off, const void* src, size_t n, const char* what) {
    return cuda_ok(cudaMemcpyAsync(c->ws + off, src, n, cudaMemcpyHostToDevice, c->stream), what);
  };
  // pageable sources: the copies are staged before the calls return
  bool ok = cuda_ok(cudaMemsetAsync(c->ws, 0, p.bytes, c->stream), "cudaMemsetAsync") &&
            up(p.off_info, t.info.data(), sizeof(ProbInfo) * t.info.size(), "cudaMemcpyAsync(problems)") &&
            up(p.off_ustart, t.ustart.data(), sizeof(long long) * t.ustart.size(), "cudaMemcpyAsync(unit starts)") &&
            up(p.off_ustartW, t.ustartW.data(), sizeof(long long) * t.ustartW.size(), "cudaMemcpyAsync(Wiener units)") &&
            up(p.off_bstartW, t.bstartW.data(), sizeof(long long) * t.bstartW.size(), "cudaMemcpyAsync(Wiener ranges)");
  c->plan.pW.info = dinfo;
  c->plan.pW.ustart = reinterpret_cast<const long long*>(c->ws + p.off_ustartW);
  c->plan.pW.bstart = reinterpret_cast<const long long*>(c->ws + p.off_bstartW);
  c->plan.pW.slots = nullptr;  // the Wiener pass sums nothing
  for (int q = 0; q < kCands && ok; ++q) {
    c->candA[q] = t.candA[q];
    c->candB[q] = t.candB[q];
    for (Partition* pp : {&c->candA[q], &c->candB[q]}) {
      pp->info = dinfo;
      pp->ustart = dustart;
    }
    c->candA[q].bstart = reinterpret_cast<const long long*>(c->ws + p.off_bstartA[q]);
    c->candB[q].bstart = reinterpret_cast<const long long*>(c->ws + p.off_bstartB[q]);
    c->candA[q].slots = reinterpret_cast<const int2*>(c->ws + p.off_slotsA[q]);
    c->candB[q].slots = reinterpret_cast<const int2*>(c->ws + p.off_slotsB[q]);
    ok = up(p.off_bstartA[q], t.bstartA[q].data(), sizeof(long long) * t.bstartA[q].size(), "cudaMemcpyAsync(ranges A)") &&
         up(p.off_bstartB[q], t.bstartB[q].data(), sizeof(long long) * t.bstartB[q].size(), "cudaMemcpyAsync(ranges B)") &&
         up(p.off_slotsA[q], t.slotsA[q].data(), sizeof(int2) * t.slotsA[q].size(), "cudaMemcpyAsync(slots A)") &&
         up(p.off_slotsB[q], t.slotsB[q].data(), sizeof(int2) * t.slotsB[q].size(), "cudaMemcpyAsync(slots B)");
  }
  if (!ok || !cuda_ok(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize")) {
    std::free(c);
    return FFCA_ERR_CUDA;
  }
  use_candidates(c, 0, 0);
  *out = c;
  return FFCA_OK;
}

ffca_status ffca_batch_iterate(ffca_batch_ctx* c, int iters, double* ll_trace) {
  if (!c || c->M < 1) return FFCA_ERR_ARG;
  return ffca_iterate(c, iters, ll_trace);
}

ffca_status ffca_batch_loglik(ffca_batch_ctx* c, double* ll) {
  if (!c || !ll || c->M < 1) return FFCA_ERR_ARG;
  ffca_status st = launch_prep(c, false);
  if (st != FFCA_OK) return st;
  FastArgs a = pass_a_args(c, 0);
  if ((st = launch(c, FFCA_KERNEL_LOGLIK, c->kern->estep_eval, stream_grid(c, a.part), stream_threads(c), a,
                   c->kern->stream_smem)) != FFCA_OK)
    return st;
  if ((st = launch(c, FFCA_KERNEL_AFINAL, c->kern->afinal_eval, finals_grid(c), 32 * kFinalWarps, a)) != FFCA_OK)
    return st;
  double* msum = reinterpret_cast<double*>(c->ws + c->plan.off_msum);
  k_mixture_sums<<<c->M, 256, 0, c->stream>>>(a.llf, c->Fm, msum);
  if (!cuda_ok(cudaGetLastError(), "k_mixture_sums") ||
      !cuda_ok(cudaMemcpyAsync(ll, msum, sizeof(double) * c->M, cudaMemcpyDeviceToHost, c->stream),
               "cudaMemcpyAsync"))
    return FFCA_ERR_CUDA;
  return read_status(c);
}

ffca_status ffca_batch_set_config(ffca_batch_ctx* c, int cand_a, int cand_b) {
  if (!c || c->M < 1 || cand_a < 0 || cand_a >= kCands || cand_b < 0 || cand_b >= kCands) return FFCA_ERR_ARG;
  use_candidates(c, cand_a, cand_b);
  return FFCA_OK;
}

int ffca_batch_config_count(void) { return kCands; }

ffca_status ffca_batch_autotune(ffca_batch_ctx* c, int rounds, int* cand_a, int* cand_b, double* ms_a,
                                double* ms_b) {
  if (!c || c->M < 1 || rounds < 1) return FFCA_ERR_ARG;
  cudaEvent_t ev[kCands][3];
  for (int q = 0; q < kCands; ++q)
    for (int e = 0; e < 3; ++e)
      if (!cuda_ok(cudaEventCreate(&ev[q][e]), "cudaEventCreate")) return FFCA_ERR_CUDA;
  double ta[kCands] = {}, tb[kCands] = {};
  ffca_status st = launch_prep(c, false);
  for (int r = 0; r < rounds && st == FFCA_OK; ++r) {
    for (int q = 0; q < kCands && st == FFCA_OK; ++q) {
      use_candidates(c, q, q);
      if (c->pmode == kPEM) {  // the EM pass (on pass A's partition) and its step; no pass B
        cudaEventRecord(ev[q][0], c->stream);
        st = launch_em_iteration(c, 0, false);
        cudaEventRecord(ev[q][1], c->stream);
        cudaEventRecord(ev[q][2], c->stream);
        continue;
      }
      // one hybrid iteration, pass A and pass B bracketed by events
      FastArgs a = pass_a_args(c, 0);
      cudaEventRecord(ev[q][0], c->stream);
      st = launch(c, FFCA_KERNEL_ESTEP, c->kern->estep_update, stream_grid(c, a.part), stream_threads(c), a,
                  c->kern->stream_smem);
      cudaEventRecord(ev[q][1], c->stream);
      FastArgs b = pass_b_args(c, 0);
      b.trace = nullptr;
      if (st == FFCA_OK)
        st = launch(c, FFCA_KERNEL_WCOV, c->kern->wcov, wcov_grid(c, b.part), wcov_threads(c), b,
                    c->kern->wcov_smem);
      cudaEventRecord(ev[q][2], c->stream);
      if (st == FFCA_OK)
        st = launch(c, FFCA_KERNEL_PSOLVE, p_step_kernel(c), p_step_grid(c, b), p_step_threads(c), b, p_step_smem(c));
    }
    if (st == FFCA_OK && !cuda_ok(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize")) st = FFCA_ERR_CUDA;
    for (int q = 0; q < kCands && st == FFCA_OK; ++q) {
      float x = 0.f, y = 0.f;
      cudaEventElapsedTime(&x, ev[q][0], ev[q][1]);
      cudaEventElapsedTime(&y, ev[q][1], ev[q][2]);
      ta[q] += x;
      tb[q] += y;
    }
  }
  for (int q = 0; q < kCands; ++q)
    for (int e = 0; e < 3; ++e) cudaEventDestroy(ev[q][e]);
  if (st != FFCA_OK) return st;
  int ba = 0, bb = 0;
  for (int q = 1; q < kCands; ++q) {
    if (ta[q] < ta[ba]) ba = q;
    if (tb[q] < tb[bb]) bb = q;
  }
  use_candidates(c, ba, bb);
  if (cand_a) *cand_a = ba;
  if (cand_b) *cand_b = bb;
  for (int q = 0; q < kCands; ++q) {
    if (ms_a) ms_a[q] = ta[q] / rounds;
    if (ms_b) ms_b[q] = tb[q] / rounds;
  }
  return read_status(c);
}

void ffca_batch_destroy(ffca_batch_ctx* c) { ffca_destroy(c); }

static_assert(FFCA_P_FIXED_POINT == kPFixedPoint && FFCA_P_GRADIENT == kPGradient &&
                  FFCA_P_NATURAL_GRADIENT == kPNatural && FFCA_P_EM == kPEM && FFCA_P_NEWTON == kPNewton,
              "the ABI's P-update codes are the kernels' modes");

ffca_status ffca_set_p_update(ffca_ctx* c, int method, double mu) {
  if (!c) return FFCA_ERR_ARG;
  if (method != FFCA_P_FIXED_POINT && method != FFCA_P_GRADIENT && method != FFCA_P_NATURAL_GRADIENT &&
      method != FFCA_P_EM && method != FFCA_P_NEWTON)
    return FFCA_ERR_ARG;
  const bool stepped = method == FFCA_P_GRADIENT || method == FFCA_P_NATURAL_GRADIENT || method == FFCA_P_NEWTON;
  if (stepped && !(std::isfinite(mu) && mu > 0.0)) return FFCA_ERR_ARG;
  if (method == FFCA_P_EM && !c->kern->estep_em) return FFCA_ERR_UNSUPPORTED;
  if (method == FFCA_P_NEWTON && !c->kern->pnewton) return FFCA_ERR_UNSUPPORTED;
  c->pmode = method;
  c->mu = stepped ? mu : 0.0;
  if (c->graph) {  // the captured launches hold the previous arguments
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return FFCA_OK;
}

ffca_status ffca_mask_init(ffca_ctx* c, const void* masks, int sweeps, double delta) {
  if (!c || sweeps < 0 || sweeps > 1000 || !(delta > 0.0 && delta <= 1.0)) return FFCA_ERR_ARG;
  if (c->d.F == 0) return FFCA_OK;
  if (!masks || (reinterpret_cast<uintptr_t>(masks) % 16) != 0) return FFCA_ERR_ARG;
  if (c->d.J > kMaskMaxJ) return FFCA_ERR_UNSUPPORTED;
  MaskArgs a;
  std::memset(&a, 0, sizeof(a));
  a.part = c->plan.pA;  // problems: frames, rows, offsets
  a.I = c->d.I;
  a.J = c->d.J;
  a.ld = c->d.ld;
  a.y = c->d.y;
  a.m = masks;
  a.v = c->d.v;
  a.lam = c->d.lambda;
  a.P = c->d.P;
  a.R = reinterpret_cast<double*>(c->ws + c->plan.off_maskR);
  a.sweeps = sweeps;
  a.delta = delta;
  a.status = c->status;
  {
    struct Range {
      Range() { nvtxRangePushA("ffca mask init"); }
      ~Range() { nvtxRangePop(); }
    } range;
    if (!cuda_ok(launch_mask_init(c->d.prec, a, c->d.F, c->stream), "launch_mask_init")) return FFCA_ERR_CUDA;
  }
  return read_status(c);
}

ffca_status ffca_set_resident(ffca_ctx* c, int enable) {
  if (!c) return FFCA_ERR_ARG;
  if (enable) {
    if (!c->kern->resident || c->max_frames > c->kern->res_max_frames) return FFCA_ERR_UNSUPPORTED;
    const size_t smem = (size_t)((c->max_frames + 3) / 4 * 4) * c->kern->res_bytes_per_frame;
    if (!cuda_ok(cudaFuncSetAttribute(c->kern->resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                 "cudaFuncSetAttribute(MaxDynamicSharedMemorySize, resident)"))
      return FFCA_ERR_CUDA;
    c->res_smem = smem;
  }
  c->resident = enable ? 1 : 0;
  if (c->graph) {  // the captured launches are the other form's
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return FFCA_OK;
}

static_assert(FFCA_FAULT_NONE == kFaultNone && FFCA_FAULT_PASS_A_NO_COPIES == kFaultPassANoCopies,
              "the ABI's fault codes are the kernels'");

ffca_status ffca_test_fault(ffca_ctx* c, int kind) {
  if (!c || (kind != FFCA_FAULT_NONE && kind != FFCA_FAULT_PASS_A_NO_COPIES)) return FFCA_ERR_ARG;
  c->fault = kind;
  if (c->graph) {  // the captured launches hold the previous arguments
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return FFCA_OK;
}

ffca_status ffca_set_graph(ffca_ctx* c, int enable) {
  if (!c) return FFCA_ERR_ARG;
  c->use_graph = enable ? 1 : 0;
  if (!enable && c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return FFCA_OK;
}

}  // extern "C"
