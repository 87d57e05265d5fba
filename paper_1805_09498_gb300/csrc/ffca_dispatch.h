// Host-side table of the compiled kernel instantiations.
#pragma once

#include <cuda_runtime.h>

namespace ffca {

// Every FastFCA-AS kernel takes one FastArgs by value.
struct FastKernels {
  int stream_smem;           // dynamic shared memory of the streaming passes
  int stream_groups;         // pipelines per CTA of the streaming passes (256 threads each)
  const void* estep_update;  // pass A with the M-step
  const void* estep_eval;    // pass A, log-likelihood only
  const void* wcov;          // pass B: weighted covariance partial sums
  const void* psolve;        // per-frequency fixed-point update of P
  const void* wiener;
  const void* prep;          // per-frequency ln|det P|^2, P^{-H}, pass-A parameters
  const void* afinal_eval;   // log-likelihood-only pass A finalise: per-frequency L2, trace
  int params_a_bytes;        // bytes per frequency of the pass-A parameter table
  int params_b_bytes;        // bytes per frequency of the pass-B parameter table
  int solve_smem;            // dynamic shared memory of psolve and prep
  int pinv_step;             // 1: the P step starts from P^{-H} (prep computes it) and leaves the next one
  const void* pgrad;         // the P step with the gradient updates in place of the fixed point
  // the normal EM update of P (nullptr where not compiled: I > 4)
  const void* estep_em;      // pass A with the EM sums (one pipeline group per CTA)
  const void* psolve_em;     // its per-problem step (no pass B)
  const void* psolve_em_wide;  // the same step with one warp per problem (I = 3, 4, 8; else nullptr)
  int em_smem;               // dynamic shared memory of estep_em
  int em_solve_smem;         // dynamic shared memory of psolve_em
  int em_nv;                 // sums per slot of estep_em
  int em_groups;             // pipeline groups per CTA of estep_em
  const void* pnewton;       // the P step with Newton's method (one block per problem)
  int newton_threads;        // its block: a warp for I <= 4, 2 I^2 + 32 threads for I = 8
  int newton_smem;           // its dynamic shared memory (the I = 8 system)
  int wcov_groups;           // pipeline groups per CTA of pass B (stream_groups: pass A)
  int wcov_smem;             // dynamic shared memory of pass B (stream_smem: pass A)
  // iterations with each problem resident in shared memory (nullptr for I > 4)
  const void* resident;
  int res_bytes_per_frame;   // shared memory per frame of a problem
  int res_max_frames;        // frames of the largest problem it takes
  const void* psolve_wide;   // the fixed-point step with one warp per problem (I = 3, 4, 8; else nullptr)
  const void* prep_wide;     // prep with one warp per problem (I = 3, 4, 8; else nullptr)
};

// prec: 0 = FP64, 1 = mixed.  nullptr if (I, J) is not compiled.
const FastKernels* fast_kernels(int prec, int I, int J);

// The three launches of the mask-based initialisation (ffca_mask.cuh) on
// stream s for `problems` problems; prec as above.
struct MaskArgs;
cudaError_t launch_mask_init(int prec, const MaskArgs& a, int problems, cudaStream_t s);

// Conventional FCA EM baseline: every kernel takes one FcaArgs by value.
struct FcaKernels {
  const void* prep;
  const void* em_update;
  const void* em_eval;
  const void* final_update;
  const void* final_eval;
  int params_bytes;  // bytes per frequency of the S_j (, S_j^{-1}) table
  int nv;            // partial sums per slot
  int em_smem;       // dynamic shared memory of the EM pass
  int final_block;   // threads per block of the finalise kernel (per frequency: 1 or a warp)
};
const FcaKernels* fca_kernels(int prec, int I, int J);

// Adjoint kernels (gradients of NLL and of the Wiener squared error): every
// kernel takes one AdjArgs by value.
struct AdjKernels {
  const void* nll;
  const void* nll_final;
  const void* se;
  const void* se_final;
  int nv_max;  // partial sums per slot (the larger loss)
};
const AdjKernels* adj_kernels(int prec, int I, int J);

#define FFCA_DECLARE_TABLE(P, I) \
  const FastKernels* fast_kernels_p##P##_i##I(int J); \
  const FcaKernels* fca_kernels_p##P##_i##I(int J); \
  const AdjKernels* adj_kernels_p##P##_i##I(int J);
FFCA_DECLARE_TABLE(0, 1)
FFCA_DECLARE_TABLE(0, 2)
FFCA_DECLARE_TABLE(0, 3)
FFCA_DECLARE_TABLE(0, 4)
FFCA_DECLARE_TABLE(0, 8)
FFCA_DECLARE_TABLE(1, 1)
FFCA_DECLARE_TABLE(1, 2)
FFCA_DECLARE_TABLE(1, 3)
FFCA_DECLARE_TABLE(1, 4)
FFCA_DECLARE_TABLE(1, 8)
#undef FFCA_DECLARE_TABLE

// The normal EM and Newton kernels of one precision, compiled in
// translation units of their own.
#define FFCA_DECLARE_ALT(P, I) \
  const void* em_estep_p##P##_i##I(int J); \
  const void* em_psolve_p##P##_i##I(int J); \
  const void* em_psolve_wide_p##P##_i##I(int J); \
  const void* newton_p##P##_i##I(int J);
FFCA_DECLARE_ALT(0, 1)
FFCA_DECLARE_ALT(0, 2)
FFCA_DECLARE_ALT(0, 3)
FFCA_DECLARE_ALT(0, 4)
FFCA_DECLARE_ALT(0, 8)
FFCA_DECLARE_ALT(1, 1)
FFCA_DECLARE_ALT(1, 2)
FFCA_DECLARE_ALT(1, 3)
FFCA_DECLARE_ALT(1, 4)
FFCA_DECLARE_ALT(1, 8)
#undef FFCA_DECLARE_ALT

}  // namespace ffca
