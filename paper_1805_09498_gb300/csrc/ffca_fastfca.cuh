// FastFCA-AS kernels (Ito & Nakatani, Sec. 4.4), except the two streaming
// passes (k_estep, k_wcov), which live in ffca_stream.cuh.
//
//   k_psolve  per frequency (one warp): V_i from the slots, then the FP64
//             fixed-point update of P(f) (K sweeps) and ln|det P(f)|^2.
//   k_wiener  x^_j = P^{-H} diag(v_j lambda_j / sigma) P^H y (Eq. MMSE0).
//   k_prep    per frequency: ln|det P|^2 and P^{-H} (FP64).
//
// Layouts: y [I][F][ld] complex (float2 or double2), v [J][F][ld] real,
// lambda [F][J][I] double, P [F][I][I] complex double row-major.  The
// streaming kernels read whole 16-byte vector units of y: two frames of a c64
// mic row, or one frame of a c128 row.
#pragma once

#include "ffca_common.cuh"

namespace ffca {

constexpr int kTraceCap = 4096;  // device-side log-likelihood trace slots
constexpr double kLnPi = 1.1447298858494002;

struct FastArgs {
  Partition part;
  int I, J, F, N, ld, K;
  const void* y;
  void* v;
  double* lam;
  double* P;
  double* part_buf;          // [F][max_slots][NV] partial sums of one pass
  unsigned* cnt;             // [F] arrival counters of that pass
  unsigned* gcnt;            // global arrival counter of that pass
  double* logdet;            // [F] ln|det P(f)|^2 of the current P
  double* llf;               // [F] per-frequency log-likelihood
  double* trace;             // [kTraceCap]
  int trace_slot;
  unsigned* status;          // [2] first error code, its frequency
  unsigned long long* ops;   // matrix inversions performed by the P update
  double* pinvH;             // [F][I][I] complex, P^{-H} (Wiener)
  void* out;                 // Wiener output [J][I][F][ld] complex
  void* tabA;                // [F] ParamsA: P(f) and Lambda(f) in the per-point precision
  void* tabB;                // [F] ParamsB: Lambda(f) in the per-point precision
  double inv_n;              // 1 / N
  double* lam_next;          // [F][J][I] the new Lambda, written during pass B, committed by k_psolve
  Partition prev_part;       // pass B reads pass A's slots: their partition
  const double* prev_buf;    // and buffer
  int pmode;                 // update of P: kPFixedPoint, kPGradient, kPNatural, kPEM or kPNewton
  double mu;                 // step size of the gradient updates
  int fault;                 // injected fault (tests of failure detection): kFault*
};

// Faults a test can inject (ffca_test_fault): with kFaultPassANoCopies the
// producers of pass A issue no copies, so that its consumers' bounded waits
// run out and latch the time-out status.
constexpr int kFaultNone = 0;
constexpr int kFaultPassANoCopies = 1;

// Updates of P: the fixed-point iteration (Eq. FPI), or K ascent steps on L2
// with the V_i of Eq. FPI held fixed (the alternatives of Sec. 4.6), of size
// mu along G / N, G = dL2/dP^* of Eq. partialP:
//   gradient  p_i <- p_i + mu ([P^{-H}]_i - V_i p_i)
//   natural   p_i <- p_i + mu (p_i - P P^H V_i p_i)   (P P^H G / N)
// The normal EM (kPEM, ffca_em.cuh) replaces the V_i of Eq. FPI by the
// M-step matrices W_i / (J N) and needs no pass B.
constexpr int kPFixedPoint = 0;
constexpr int kPGradient = 1;
constexpr int kPNatural = 2;
constexpr int kPEM = 3;
constexpr int kPNewton = 4;  // K Newton steps of size mu (ffca_newton.cuh)

// Matrix inversions per problem of one P update: (I+1) K for the fixed
// point (Sec. 4.5) and for the normal EM (the same map on other matrices),
// one P^{-H} per gradient step, none for the natural gradient, two per
// Newton step (P and the 2 I^2 system).
__device__ inline unsigned long long p_update_inversions(const FastArgs& a, int I) {
  if (a.pmode == kPFixedPoint || a.pmode == kPEM) return (unsigned long long)(I + 1) * a.K;
  if (a.pmode == kPGradient) return (unsigned long long)a.K;
  if (a.pmode == kPNewton) return 2ull * a.K;
  return 0ull;
}

// Per-frequency parameters in the per-point precision T, laid out as they
// travel to the streaming kernels (one bulk copy per tile, 16-byte padded).
// Pass A's record holds P(f) and Lambda(f).  With DUP every value would be
// stored twice, P as (re, re, im, im) per entry and Lambda as (l, l), for
// loading packed f32x2 operands directly; measured slower for pass A at
// I = 8 (109 us against 99 us with single values), so it is off.
template <typename T, int I, int J>
struct ParamsA {
  static constexpr bool DUP = false;
  static constexpr int NP = (DUP ? 4 : 2) * I * I;  // P values
  static constexpr int NL = (DUP ? 2 : 1) * J * I;  // Lambda values
  T v[NP + NL];
  static constexpr int BYTES = (int)((sizeof(T) * (NP + NL) + 15) / 16 * 16);
  __device__ T pre(int r, int c) const { return DUP ? v[4 * (r * I + c)] : v[r * I + c]; }
  __device__ T pim(int r, int c) const { return DUP ? v[4 * (r * I + c) + 2] : v[I * I + r * I + c]; }
  __device__ T lam(int j, int i) const { return DUP ? v[NP + 2 * (j * I + i)] : v[NP + j * I + i]; }
  __device__ void set_p(int r, int c, T re, T im) {
    if constexpr (DUP) {
      T* q = v + 4 * (r * I + c);
      q[0] = re;
      q[1] = re;
      q[2] = im;
      q[3] = im;
    } else {
      v[r * I + c] = re;
      v[I * I + r * I + c] = im;
    }
  }
  __device__ void set_lam(int j, int i, T l) {
    if constexpr (DUP) {
      v[NP + 2 * (j * I + i)] = l;
      v[NP + 2 * (j * I + i) + 1] = l;
    } else {
      v[NP + j * I + i] = l;
    }
  }
};
// Pass A's record of problem f for a J known only at run time (the layout
// of ParamsA<T, I, J> with single values): P's real parts, its imaginary
// parts, then Lambda.
template <typename T, int I>
struct ParamsARun {
  T* v;
  __device__ ParamsARun(void* tab, int J, int f) {
    const size_t bytes = (sizeof(T) * (2 * I * I + (size_t)J * I) + 15) / 16 * 16;
    v = reinterpret_cast<T*>(static_cast<char*>(tab) + (size_t)f * bytes);
  }
  __device__ void set_p(int r, int c, T re, T im) {
    v[r * I + c] = re;
    v[I * I + r * I + c] = im;
  }
  __device__ void set_lam(int j, int i, T l) { v[2 * I * I + j * I + i] = l; }
};
static_assert(!ParamsA<float, 1, 1>::DUP, "ParamsARun assumes single values");

template <typename T, int I, int J>
struct ParamsB {  // pass B: the new Lambda(f)
  T lam[J][I];
  static constexpr int BYTES = (int)((sizeof(T) * J * I + 15) / 16 * 16);
};
template <typename T, int I, int J>
__device__ inline ParamsA<T, I, J>* tab_a(const FastArgs& a, int f) {
  return reinterpret_cast<ParamsA<T, I, J>*>(static_cast<char*>(a.tabA) + (size_t)f * ParamsA<T, I, J>::BYTES);
}
template <typename T, int I, int J>
__device__ inline ParamsB<T, I, J>* tab_b(const FastArgs& a, int f) {
  return reinterpret_cast<ParamsB<T, I, J>*>(static_cast<char*>(a.tabB) + (size_t)f * ParamsB<T, I, J>::BYTES);
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using Y = float4;  // two c64 frames
  using V = float2;  // two real frames
  static constexpr int FU = 2;
};
template <>
struct Vec<double> {
  using Y = double2;  // one c128 frame
  using V = double;   // one real frame
  static constexpr int FU = 1;
};

__device__ inline cpx<float> yframe(const float4& u, int e) {
  return e == 0 ? mk(u.x, u.y) : mk(u.z, u.w);
}
__device__ inline cpx<double> yframe(const double2& u, int) { return mk(u.x, u.y); }
__device__ inline float vframe(const float2& u, int e) { return e == 0 ? u.x : u.y; }
__device__ inline double vframe(double u, int) { return u; }
__device__ inline void vset(float2& u, int e, float x) {
  if (e == 0) u.x = x; else u.y = x;
}
__device__ inline void vset(double& u, int, double x) { u = x; }
__device__ inline void yset(float4& u, int e, cpx<float> z) {
  if (e == 0) { u.x = z.re; u.y = z.im; } else { u.z = z.re; u.w = z.im; }
}
__device__ inline void yset(double2& u, int, cpx<double> z) { u.x = z.re; u.y = z.im; }

constexpr int kUnits = 2;  // vector units per thread per loop trip

// Sum the partial slots of frequency f for value t in slot order (deterministic).
__device__ inline double sum_slots(const double* part_buf, int f, int nslots, int max_slots,
                                   int NV, int t) {
  const double* p = part_buf + ((size_t)f * max_slots) * NV + t;
  double s = 0.0;
  for (int k = 0; k < nslots; ++k) s += __ldcg(p + (size_t)k * NV);
  return s;
}

// Sum of the n values v[0..n) in a fixed order by one warp (lane l takes
// v[l + 32 u] of each round of 512, all 16 loads of a round in flight at
// once; a fixed tree over u, then over the lanes).  Returned in every lane.
__device__ inline double warp_sum_fixed(const double* v, int n) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
  for (int b = 0; b < n; b += 512) {
    double s[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = b + lane + 32 * u;
      s[u] = k < n ? __ldcg(v + k) : 0.0;
    }
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) s[u] += s[u + w];
    t += s[0];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

// Sum of the per-frequency log-likelihoods into the trace slot (one warp).
__device__ inline void finalize_trace(const FastArgs& a) {
  const double t = warp_sum_fixed(a.llf, a.F);
  if ((threadIdx.x & 31) == 0) a.trace[a.trace_slot] = t;
}

// With a trace, the P step is launched with one block (one warp) beyond its
// problems' blocks: that block sums the problems' log-likelihoods of the
// state entering the iteration (complete since pass B) into the trace slot,
// beside the problems' blocks instead of after them.
__device__ inline bool trace_block(const FastArgs& a) {
  if (!a.trace || blockIdx.x != gridDim.x - 1) return false;
  finalize_trace(a);
  return true;
}

// -------------------------------------------------------------- pass A finalise
// One warp per frequency, after pass A: sum the slots (FP64, slot order) into
// the new Lambda(f) (Eq. Lambdaupdate: lambda_ji I sum_n t_ji / s_j / N, see
// k_estep; used with UPDATE only) and the frequency's log-likelihood (Eq. L2);
// the last warp to finish adds the frequencies' log-likelihoods into the
// trace.  Inside an iteration pass B's producer does this work instead; the
// log-likelihood-only pass uses this kernel.
constexpr int kFinalWarps = 4;

template <typename T, int I, int J, bool UPDATE>
__global__ void __launch_bounds__(32 * kFinalWarps) k_afinal(FastArgs a) {
  constexpr int NA = UPDATE ? J * I : 0;
  constexpr int NV = NA + 2;
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * kFinalWarps + (threadIdx.x >> 5);
  if (f >= a.F) return;  // whole warps only
  const Partition pt = a.part;
  const int ns = pt.nslots(f);
  for (int q = lane; q < NA; q += 32) {
    const int j = q / I, i = q % I;
    const double tot = sum_slots(a.part_buf, f, ns, pt.max_slots, NV, q);
    double* lp = a.lam + (size_t)f * J * I + q;
    const double lnew = *lp * ((double)I * pt.inv_n(f)) * tot;
    if (!(lnew > 0.0) || !isfinite(lnew)) raise_status(a.status, kDevNonfinite, f);
    *lp = lnew;
    tab_a<T, I, J>(a, f)->set_lam(j, i, (T)lnew);
    tab_b<T, I, J>(a, f)->lam[j][i] = (T)lnew;
  }
  if (lane == NA % 32) {
    const double quad = sum_slots(a.part_buf, f, ns, pt.max_slots, NV, NA);
    const double lg2 = sum_slots(a.part_buf, f, ns, pt.max_slots, NV, NA + 1);
    const int n = pt.frames(f);
    const double lf = -(double)I * n * kLnPi + (double)n * a.logdet[f] - quad - 0.69314718055994530942 * lg2;
    if (!isfinite(lf)) raise_status(a.status, kDevNonfinite, f);
    a.llf[f] = lf;
    __threadfence();
  }
  __syncwarp();
  unsigned last = 0;
  if (lane == 0) {
    last = atomicAdd(a.gcnt, 1u) == (unsigned)a.F - 1;
    if (last) *a.gcnt = 0u;  // ready for the next launch
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    finalize_trace(a);
  }
}

// -------------------------------------------------------------- P update
// Packed Hermitian V_i: I real diagonal entries, then (re, im) of the
// entries above the diagonal in row order; I^2 reals per i.
template <int I>
__device__ inline void unpack_herm(const double* src, cpx<double> (&V)[I][I]) {
  int m = I;
#pragma unroll
  for (int r = 0; r < I; ++r) {
    V[r][r] = mk(src[r], 0.0);
#pragma unroll
    for (int c = r + 1; c < I; ++c) {
      V[r][c] = mk(src[m], src[m + 1]);
      V[c][r] = mk(src[m], -src[m + 1]);
      m += 2;
    }
  }
}

// -------------------------------------------------------------- P solve
// The per-frequency FP64 kernels put 32 / I frequencies in one warp, lane
// (g, i) owning column i of frequency g: FP64 throughput on this part is a
// small fraction of FP32 and a warp instruction costs the same with 3 or 32
// active lanes, so filling the lanes is what makes these kernels fast.
template <int I>
struct Lanes {
  static constexpr int G = 32 / I;  // frequencies per warp
};

__device__ inline cpx<double> shfl_c(cpx<double> z, int src) {
  return mk(__shfl_sync(0xffffffffu, z.re, src), __shfl_sync(0xffffffffu, z.im, src));
}

// Gather the full P of this lane's frequency from the I lanes that own its
// columns (lane g*I + c holds column c).
template <int I>
__device__ inline void gather_columns(const cpx<double> (&col)[I], int g, cpx<double> (&A)[I][I]) {
#pragma unroll
  for (int c = 0; c < I; ++c)
#pragma unroll
    for (int r = 0; r < I; ++r) A[r][c] = shfl_c(col[r], g * I + c);
}

// After pass B, per frequency: commit the new Lambda (computed during pass B)
// to lambda and the pass-A table; sum pass B's slots into V_i (FP64, slot
// order); the fixed-point update of P(f) (Eq. FPI, K sweeps, all columns from
// the same P^{-H}) into P and the pass-A table; finally the last warp adds
// the frequencies' log-likelihoods (also written during pass B) into the
// trace.  FP64 latency on this part is long (an FMA ~64 cycles, a division
// ~350) and its throughput low, so the kernel keeps its dependency chains
// short and its operation count small: the inverses by cofactors
// (independent, shallow products; 4 x 4 through shared 2 x 2 minors) with one
// division per sweep, register-only indexing.  It ends with ln|det P|^2 of
// the new P, which the next iteration's L2 needs (Eq. L2).
// GRAD selects the gradient updates (a separate kernel, so that the
// fixed-point one keeps its registers).
template <typename T, int I, int J, bool GRAD = false>
__global__ void __launch_bounds__(32) k_psolve(FastArgs a) {
  constexpr int G = Lanes<I>::G;
  constexpr int NV = I * I * I;
  if (trace_block(a)) return;
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f0 = blockIdx.x * G + g;
  const bool active = g < G && f0 < a.F;
  const int f = active ? f0 : 0;  // idle lanes shadow frequency 0 and write nothing
  const Partition pt = a.part;
  const int ns = pt.nslots(f);

  if (active && a.lam_next) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const double l = a.lam_next[(size_t)f * J * I + j * I + i];
      a.lam[(size_t)f * J * I + j * I + i] = l;
      ta->set_lam(j, i, (T)l);
    }
  }

  cpx<double> V[I][I];
  {
    // slot by slot, all I^2 values of V_i at once: the loads of a slot are in flight together
    double pk[I * I];
#pragma unroll
    for (int m = 0; m < I * I; ++m) pk[m] = 0.0;
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV + i * I * I;
    for (int k = 0; k < ns; ++k)
#pragma unroll
      for (int m = 0; m < I * I; ++m) pk[m] += __ldcg(base + (size_t)k * NV + m);
#pragma unroll
    for (int m = 0; m < I * I; ++m) pk[m] *= pt.inv_n(f);
    unpack_herm<I>(pk, V);
  }
  bool bad = false;
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) bad |= !isfinite(V[r][c].re) || !isfinite(V[r][c].im);
  if (active && bad) raise_status(a.status, kDevNonfinite, f);

  cpx<double> A[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c)
      A[r][c] = mk(a.P[((size_t)f * I * I + r * I + c) * 2], a.P[((size_t)f * I * I + r * I + c) * 2 + 1]);

  bool singular = false;
  if constexpr (GRAD) {
    // the gradient steps: V_i is multiplied, not inverted
    for (int sweep = 0; sweep < a.K; ++sweep) {
      cpx<double> p[I], w[I], col[I];
#pragma unroll
      for (int r = 0; r < I; ++r) {
        p[r] = A[r][0];
#pragma unroll
        for (int c = 1; c < I; ++c)
          if (c == i) p[r] = A[r][c];
      }
#pragma unroll
      for (int r = 0; r < I; ++r) {  // w = V_i p_i
        w[r] = mk(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < I; ++c) cfma(w[r], V[r][c], p[c]);
      }
      if (a.pmode == kPGradient) {  // [P^{-H}]_{ri} = conj(C_P[r][i] / det P)
        cpx<double> C[I][I];
        const cpx<double> detP = cofactors<I>(A, C);
        const double d2 = cabs2(detP);
        singular |= !(d2 > 0.0) || !isfinite(d2);
        const double inv = 1.0 / d2;
        const cpx<double> rdet = mk(detP.re * inv, -detP.im * inv);
#pragma unroll
        for (int r = 0; r < I; ++r) {
          cpx<double> cri = C[r][0];
#pragma unroll
          for (int c = 1; c < I; ++c)
            if (c == i) cri = C[r][c];
          const cpx<double> x = cconj(cmul(cri, rdet));
          col[r] = mk(p[r].re + a.mu * (x.re - w[r].re), p[r].im + a.mu * (x.im - w[r].im));
        }
      } else {  // natural: P (P^H w) with column k of P in A[., k]
        cpx<double> u[I];
#pragma unroll
        for (int r = 0; r < I; ++r) u[r] = mk(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < I; ++k) {
          cpx<double> ck = mk(0.0, 0.0);
#pragma unroll
          for (int q = 0; q < I; ++q) cfma(ck, cconj(A[q][k]), w[q]);
#pragma unroll
          for (int r = 0; r < I; ++r) cfma(u[r], A[r][k], ck);
        }
#pragma unroll
        for (int r = 0; r < I; ++r)
          col[r] = mk(p[r].re + a.mu * (p[r].re - u[r].re), p[r].im + a.mu * (p[r].im - u[r].im));
      }
      gather_columns<I>(col, g, A);
    }
  } else {
    // V_i^{-1} = adj(V_i) / det V_i with adj(V) = C_V^T (cofactors, once per
    // iteration), so that one division per sweep remains on the critical path:
    //   p_i = V_i^{-1} [P^{-H}]_i = adj(V_i) conj(C_P[., i]) / (det V_i conj(det P))
    // since [P^{-H}]_{r i} = conj((P^{-1})_{i r}) = conj(C_P[r][i]) / conj(det P).
    cpx<double> CV[I][I];
    const double detV = cofactors<I>(V, CV).re;  // real for Hermitian V
    double diagprod = 1.0;
#pragma unroll
    for (int r = 0; r < I; ++r) diagprod *= V[r][r].re;
    // Hadamard: 0 < det V <= prod V_rr for positive definite V; a ratio at
    // rounding level means rank deficiency
    singular = !(detV > kCholRtol * diagprod) || !isfinite(detV);
    for (int sweep = 0; sweep < a.K; ++sweep) {
      cpx<double> C[I][I];
      const cpx<double> detP = cofactors<I>(A, C);
      cpx<double> num[I];
#pragma unroll
      for (int r = 0; r < I; ++r) {
        cpx<double> s = mk(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < I; ++q) {
          cpx<double> cqi = C[q][0];  // column i of C_P, selected by predicate
#pragma unroll
          for (int c = 1; c < I; ++c)
            if (c == i) cqi = C[q][c];
          cfma(s, CV[q][r], cconj(cqi));  // adj(V)_{rq} = CV_{qr}
        }
        num[r] = s;
      }
      const cpx<double> den = mk(detV * detP.re, -detV * detP.im);  // det V conj(det P)
      const double d2 = cabs2(den);
      singular |= !(cabs2(detP) > 0.0) || !isfinite(d2);
      const double inv = 1.0 / d2;
      const cpx<double> rden = mk(den.re * inv, -den.im * inv);
      cpx<double> col[I];
#pragma unroll
      for (int r = 0; r < I; ++r) col[r] = cmul(num[r], rden);
      gather_columns<I>(col, g, A);
    }
  }
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int r = 0; r < I; ++r) {
      cpx<double> ari = A[r][0];
#pragma unroll
      for (int c = 1; c < I; ++c)
        if (c == i) ari = A[r][c];
      a.P[((size_t)f * I * I + r * I + i) * 2] = ari.re;
      a.P[((size_t)f * I * I + r * I + i) * 2 + 1] = ari.im;
      ta->set_p(r, i, (T)ari.re, (T)ari.im);
    }
    if (singular) raise_status(a.status, kDevSingular, f);
    if (i == 0) {
      atomicAdd(a.ops, p_update_inversions(a, I));
      const double d2 = cabs2(determinant<I>(A));
      if (!(d2 > 0.0) || !isfinite(d2)) raise_status(a.status, kDevSingular, f);
      a.logdet[f] = log(d2);
    }
  }
}

// -------------------------------------------------------------- prep
// ln|det P|^2 and, if requested, P^{-H} of the current P (FP64, cofactors;
// lane (g, i) computes column i of P^{-H} of frequency g), and the pass-A
// parameter table from the current P and Lambda.
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_prep(FastArgs a) {
  constexpr int G = Lanes<I>::G;
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f = blockIdx.x * G + g;
  if (g >= G || f >= a.F) return;
  cpx<double> A[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c)
      A[r][c] = mk(a.P[((size_t)f * I * I + r * I + c) * 2], a.P[((size_t)f * I * I + r * I + c) * 2 + 1]);
  ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
  for (int r = 0; r < I; ++r) {
    ta->set_p(r, i, (T)A[r][i].re, (T)A[r][i].im);
  }
#pragma unroll
  for (int j = 0; j < J; ++j) ta->set_lam(j, i, (T)a.lam[(size_t)f * J * I + j * I + i]);
  cpx<double> C[I];
  const cpx<double> det = column_cofactors<I>(A, i, C);
  const double d2 = cabs2(det);
  const bool ok = d2 > 0.0 && isfinite(d2);
  if (!ok) raise_status(a.status, kDevSingular, f);
  if (i == 0) a.logdet[f] = log(d2);
  if (a.pinvH) {
    const double inv = 1.0 / d2;
    const cpx<double> rdet = mk(det.re * inv, -det.im * inv);
#pragma unroll
    for (int r = 0; r < I; ++r) {  // (P^{-H})_{r i} = conj((P^{-1})_{i r}) = conj(C_ri / det)
      const cpx<double> q = cconj(cmul(C[r], rdet));
      a.pinvH[((size_t)f * I * I + r * I + i) * 2] = q.re;
      a.pinvH[((size_t)f * I * I + r * I + i) * 2 + 1] = q.im;
    }
  }
}

// -------------------------------------------------------------- Wiener
template <typename T, int I, int J>
__global__ void __launch_bounds__(kBlock) k_wiener(FastArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  constexpr int FU = Vec<T>::FU;
  __shared__ double sP[I][I][2], sQ[I][I][2];
  __shared__ double sLam[J][I];

  const Partition pt = a.part;
  const long long u0 = pt.block_start(blockIdx.x);
  const long long u1 = pt.block_start(blockIdx.x + 1);
  const long long row = a.ld / FU;

  // the block's unit range, problem by problem (a problem's units cover all
  // ld_m frames of its rows, padding included)
  for (long long u = u0; u < u1;) {
    const int f = pt.problem_of(u);
    const long long us = pt.start(f);
    const int k0 = (int)(u - us);
    const int k1 = (int)(min(pt.start(f + 1), u1) - us);
    const int Np = pt.frames(f);
    const long long rlen = pt.row_len(f, row * FU) / FU;  // units per row of the problem's blocks
    const long long off = pt.frame_off(f) / FU;
    const long long r0 = (long long)pt.freq(f) * rlen;
    // rows: mic m at I Fm off + m Fm rlen + r0, source j at J Fm off + j Fm rlen + r0,
    // output (j, r) at J I Fm off + (j I + r) Fm rlen + r0
    const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y) + (size_t)I * pt.Fm * off + r0;
    const VV* __restrict__ v = reinterpret_cast<const VV*>(a.v) + (size_t)J * pt.Fm * off + r0;
    VY* __restrict__ out = reinterpret_cast<VY*>(a.out) + (size_t)J * I * pt.Fm * off + r0;
    const size_t rstr = (size_t)pt.Fm * rlen;  // stride between the problem's rows
    __syncthreads();
    if (threadIdx.x < I * I) {
      const int r = threadIdx.x / I, c = threadIdx.x % I;
      sP[r][c][0] = a.P[((size_t)f * I * I + threadIdx.x) * 2];
      sP[r][c][1] = a.P[((size_t)f * I * I + threadIdx.x) * 2 + 1];
      sQ[r][c][0] = a.pinvH[((size_t)f * I * I + threadIdx.x) * 2];
      sQ[r][c][1] = a.pinvH[((size_t)f * I * I + threadIdx.x) * 2 + 1];
    }
    if (threadIdx.x < J * I) sLam[threadIdx.x / I][threadIdx.x % I] = a.lam[(size_t)f * J * I + threadIdx.x];
    __syncthreads();
    cpx<T> Pc[I][I], Q[I][I];
    T lam[J][I];
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) {
        Pc[r][c] = mk<T>((T)sP[r][c][0], (T)sP[r][c][1]);
        Q[r][c] = mk<T>((T)sQ[r][c][0], (T)sQ[r][c][1]);
      }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int i = 0; i < I; ++i) lam[j][i] = (T)sLam[j][i];

    for (int k = k0 + threadIdx.x; k < k1; k += kBlock) {
      VY yu[I];
      VV vu[J];
#pragma unroll
      for (int m = 0; m < I; ++m) yu[m] = y[m * rstr + k];
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = v[j * rstr + k];
      VY o[J][I];
#pragma unroll
      for (int e = 0; e < FU; ++e) {
        const bool valid = k * FU + e < Np;
        cpx<T> yt[I];
#pragma unroll
        for (int i = 0; i < I; ++i) {
          cpx<T> s = mk<T>(0, 0);
#pragma unroll
          for (int m = 0; m < I; ++m) cfmac(s, Pc[m][i], yframe(yu[m], e));
          yt[i] = s;
        }
        T rs[I];
#pragma unroll
        for (int i = 0; i < I; ++i) {
          T s = vframe(vu[0], e) * lam[0][i];
#pragma unroll
          for (int j = 1; j < J; ++j) s = fma(vframe(vu[j], e), lam[j][i], s);
          rs[i] = recip(s);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
          cpx<T> z[I];
#pragma unroll
          for (int i = 0; i < I; ++i) z[i] = cscale(yt[i], vframe(vu[j], e) * lam[j][i] * rs[i]);
#pragma unroll
          for (int r = 0; r < I; ++r) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int i = 0; i < I; ++i) cfma(s, Q[r][i], z[i]);
            yset(o[j][r], e, valid ? s : mk<T>(0, 0));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j)
#pragma unroll
        for (int r = 0; r < I; ++r) out[(j * I + r) * rstr + k] = o[j][r];
    }
    u += k1 - k0;
  }
}

}  // namespace ffca
