// Explicit instantiations of the FastFCA-AS kernels (FFCA_PART 0), of the
// conventional FCA kernels (FFCA_PART 1), of the adjoint kernels
// (FFCA_PART 2), of the normal EM update of P (FFCA_PART 3) or of Newton's
// method for P (FFCA_PART 4) for one precision and one microphone count,
// J = 1..6 (parts 3 and 4: I <= 4).
// Compiled once per (FFCA_PART, FFCA_PREC, FFCA_I).
#include "ffca_adjoint.cuh"
#include "ffca_big.cuh"
#include "ffca_dispatch.h"
#include "ffca_em.cuh"
#include "ffca_fca.cuh"
#include "ffca_fca_big.cuh"
#include "ffca_newton.cuh"
#include "ffca_psolve_wide.cuh"
#include "ffca_resident.cuh"
#include "ffca_stream.cuh"

#ifndef FFCA_PREC
#error "FFCA_PREC must be defined (0 = FP64, 1 = mixed)"
#endif
#ifndef FFCA_I
#error "FFCA_I must be defined"
#endif
#ifndef FFCA_PART
#error "FFCA_PART must be defined (0 = FastFCA-AS, 1 = FCA, 2 = adjoint, 3 = normal EM, 4 = Newton)"
#endif

#define FFCA_CAT2(a, b, c, d) a##b##c##d
#define FFCA_CAT(a, b, c, d) FFCA_CAT2(a, b, c, d)

namespace ffca {

#if FFCA_PREC == 0
using Real = double;
#else
using Real = float;
#endif

#if FFCA_PART == 0
// The P step by Gauss-Jordan and LDL^H (k_psolve_ldl, which carries P^{-H}
// from one step to the next) from FFCA_LDL_MIN_I microphones up; below it
// the cofactor forms of k_psolve.  At I = 3, 4 and 8 the fixed point and
// prep of up to about a thousand problems (ffca_api.cu) run k_psolve_wide
// and k_prep_wide (one warp per problem, the same P^{-H} bits).
#ifndef FFCA_LDL_MIN_I
#define FFCA_LDL_MIN_I 3
#endif
template <int J>
static const FastKernels* table_entry() {
  constexpr bool BIG = FFCA_I > 4;            // per-point parameters read from the stage, per-source Wiener
  constexpr bool LDL = FFCA_I >= FFCA_LDL_MIN_I;
  const void* psolve;
  const void* pgrad;
  const void* prep;
  const void* wiener;
  if constexpr (LDL) {
    psolve = (const void*)k_psolve_ldl<Real, FFCA_I, J>;
    pgrad = (const void*)k_psolve_ldl<Real, FFCA_I, J, true>;
    prep = (const void*)k_prep_gj<Real, FFCA_I, J>;
  } else {
    psolve = (const void*)k_psolve<Real, FFCA_I, J>;
    pgrad = (const void*)k_psolve<Real, FFCA_I, J, true>;
    prep = (const void*)k_prep<Real, FFCA_I, J>;
  }
  const void* psolve_wide = nullptr;
  const void* prep_wide = nullptr;
  if constexpr (FFCA_I == 3 || FFCA_I == 4 || FFCA_I == 8) {
    psolve_wide = (const void*)k_psolve_wide<Real, FFCA_I, J>;
    prep_wide = (const void*)k_prep_wide<Real, FFCA_I, J>;
  }
  if constexpr (BIG) wiener = (const void*)k_wiener_big<Real, FFCA_I, J>;
  else wiener = (const void*)k_wiener<Real, FFCA_I, J>;
  // the normal EM and Newton kernels are compiled in translation units of
  // their own (FFCA_PART 3 and 4), so that they build in parallel
  const void* estep_em = nullptr;
  const void* psolve_em = nullptr;
  const void* pnewton = FFCA_CAT(newton_p, FFCA_PREC, _i, FFCA_I)(J);
  const int newton_threads = FFCA_I > 4 ? NewtonBig<FFCA_I>::THREADS : 32;
  const int newton_smem = FFCA_I > 4 ? NewtonBig<FFCA_I>::BYTES : 0;
  int em_smem = 0, em_solve_smem = 0, em_nv = 0, em_groups = 1;
  const void* resident = nullptr;
  int res_bpf = 0, res_max = 0;
  estep_em = FFCA_CAT(em_estep_p, FFCA_PREC, _i, FFCA_I)(J);
  psolve_em = FFCA_CAT(em_psolve_p, FFCA_PREC, _i, FFCA_I)(J);
  const void* psolve_em_wide = FFCA_CAT(em_psolve_wide_p, FFCA_PREC, _i, FFCA_I)(J);
  em_groups = EmGroups<Real, FFCA_I, J>::value;
  em_smem = em_groups * Tile<Real, FFCA_I, J, EmGroups<Real, FFCA_I, J>::value>::GROUP;
  em_solve_smem = EmShape<FFCA_I, J>::SMEM;
  em_nv = EmShape<FFCA_I, J>::NV;
  resident = (const void*)k_resident<Real, FFCA_I, J>;
  res_bpf = ResShape<Real, FFCA_I, J>::BYTES_PER_FRAME;
  res_max = ResShape<Real, FFCA_I, J>::max_frames();
  static const FastKernels k = {
      Tile<Real, FFCA_I, J>::G * Tile<Real, FFCA_I, J>::GROUP,
      StreamGroups<Real, FFCA_I, J>::value,
      (const void*)k_estep<Real, FFCA_I, J, true>,
      (const void*)k_estep<Real, FFCA_I, J, false>,
      (const void*)k_wcov<Real, FFCA_I, J>,
      psolve,
      wiener,
      prep,
      (const void*)k_afinal<Real, FFCA_I, J, false>,
      ParamsA<Real, FFCA_I, J>::BYTES,
      ParamsB<Real, FFCA_I, J>::BYTES,
      LDL ? BigLane<FFCA_I>::SMEM : 0,
      LDL ? 1 : 0,
      pgrad,
      estep_em,
      psolve_em,
      psolve_em_wide,
      em_smem,
      em_solve_smem,
      em_nv,
      em_groups,
      pnewton,
      newton_threads,
      newton_smem,
      WcovGroups<Real, FFCA_I, J>::value,
      WcovGroups<Real, FFCA_I, J>::value * Tile<Real, FFCA_I, J, WcovGroups<Real, FFCA_I, J>::value>::GROUP,
      resident,
      res_bpf,
      res_max,
      psolve_wide,
      prep_wide,
  };
  return &k;
}

#endif

#if FFCA_PART == 1
template <int J>
static const FcaKernels* fca_entry() {
  if constexpr (FFCA_I > 4) {  // the rearranged form (one warp per source, per-frequency products)
    using B = FcaBig<Real, FFCA_I, J>;
    static const FcaKernels k = {
        (const void*)k_fca_prep_big<Real, FFCA_I, J>,
        (const void*)k_fca_em_big<Real, FFCA_I, J, true>,
        (const void*)k_fca_em_big<Real, FFCA_I, J, false>,
        (const void*)k_fca_final_big<Real, FFCA_I, J, true>,
        (const void*)k_fca_final_big<Real, FFCA_I, J, false>,
        FcaParamsBig<Real, FFCA_I, J>::BYTES,
        B::NV,
        B::SMEM,
        128,
    };
    return &k;
  } else {
    static const FcaKernels k = {
        (const void*)k_fca_prep<Real, FFCA_I, J>,
        (const void*)k_fca_em<Real, FFCA_I, J, true>,
        (const void*)k_fca_em<Real, FFCA_I, J, false>,
        (const void*)k_fca_final<Real, FFCA_I, J, true>,
        (const void*)k_fca_final<Real, FFCA_I, J, false>,
        FcaParams<Real, FFCA_I, J>::BYTES,
        J * FFCA_I * FFCA_I + 1,
        0,
        1,
    };
    return &k;
  }
}

#endif

#if FFCA_PART == 2
template <int J>
static const AdjKernels* adj_entry() {
#if FFCA_I > 4
  static const AdjKernels k = {
      (const void*)k_adj_big<Real, FFCA_I, J, false>,
      (const void*)k_adj_final<Real, FFCA_I, J, false>,
      (const void*)k_adj_big<Real, FFCA_I, J, true>,
      (const void*)k_adj_final<Real, FFCA_I, J, true>,
      AdjShape<FFCA_I, J, false>::NV,
  };
#else
  static const AdjKernels k = {
      (const void*)k_adj<Real, FFCA_I, J, false>,
      (const void*)k_adj_final<Real, FFCA_I, J, false>,
      (const void*)k_adj<Real, FFCA_I, J, true>,
      (const void*)k_adj_final<Real, FFCA_I, J, true>,
      AdjShape<FFCA_I, J, false>::NV,
  };
#endif
  return &k;
}

#endif


#if FFCA_PART == 0
const FastKernels* FFCA_CAT(fast_kernels_p, FFCA_PREC, _i, FFCA_I)(int J) {
  switch (J) {
    case 1: return table_entry<1>();
    case 2: return table_entry<2>();
    case 3: return table_entry<3>();
    case 4: return table_entry<4>();
    case 5: return table_entry<5>();
    case 6: return table_entry<6>();
    default: return nullptr;
  }
}

#endif

#if FFCA_PART == 1
const FcaKernels* FFCA_CAT(fca_kernels_p, FFCA_PREC, _i, FFCA_I)(int J) {
  switch (J) {
    case 1: return fca_entry<1>();
    case 2: return fca_entry<2>();
    case 3: return fca_entry<3>();
    case 4: return fca_entry<4>();
    case 5: return fca_entry<5>();
    case 6: return fca_entry<6>();
    default: return nullptr;
  }
}
#endif

#if FFCA_PART == 2
const AdjKernels* FFCA_CAT(adj_kernels_p, FFCA_PREC, _i, FFCA_I)(int J) {
  switch (J) {
    case 1: return adj_entry<1>();
    case 2: return adj_entry<2>();
    case 3: return adj_entry<3>();
    case 4: return adj_entry<4>();
    case 5: return adj_entry<5>();
    case 6: return adj_entry<6>();
    default: return nullptr;
  }
}
#endif

#if FFCA_PART == 3
// kind 0: the EM pass; 1: the packed EM step; 2: the wide EM step (I = 3, 4, 8)
template <int J>
static const void* em_kernel(int kind) {
  if (kind == 1) return (const void*)k_psolve_em<Real, FFCA_I, J>;
  if (kind == 2) {
    if constexpr (FFCA_I == 3 || FFCA_I == 4 || FFCA_I == 8) return (const void*)k_psolve_em_wide<Real, FFCA_I, J>;
    return nullptr;
  }
#if FFCA_I > 4
  return (const void*)k_estep_em_big<Real, FFCA_I, J>;
#else
  return (const void*)k_estep<Real, FFCA_I, J, true, true>;
#endif
}
static const void* em_select(int J, int kind) {
  switch (J) {
    case 1: return em_kernel<1>(kind);
    case 2: return em_kernel<2>(kind);
    case 3: return em_kernel<3>(kind);
    case 4: return em_kernel<4>(kind);
    case 5: return em_kernel<5>(kind);
    case 6: return em_kernel<6>(kind);
    default: return nullptr;
  }
}
const void* FFCA_CAT(em_estep_p, FFCA_PREC, _i, FFCA_I)(int J) { return em_select(J, 0); }
const void* FFCA_CAT(em_psolve_p, FFCA_PREC, _i, FFCA_I)(int J) { return em_select(J, 1); }
const void* FFCA_CAT(em_psolve_wide_p, FFCA_PREC, _i, FFCA_I)(int J) { return em_select(J, 2); }
#endif

#if FFCA_PART == 4
// one kernel for every J (J is read from the arguments)
const void* FFCA_CAT(newton_p, FFCA_PREC, _i, FFCA_I)(int J) {
#if FFCA_I > 4
  return (J >= 1 && J <= 6) ? (const void*)k_psolve_newton_big<Real, FFCA_I> : nullptr;
#else
  return (J >= 1 && J <= 6) ? (const void*)k_psolve_newton<Real, FFCA_I> : nullptr;
#endif
}
#endif

}  // namespace ffca
