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
};

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

// The last frequency finaliser adds the per-frequency log-likelihoods in
// frequency order (one warp, fixed tree) into the trace slot.
__device__ inline void finalize_trace(const FastArgs& a) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int f = threadIdx.x; f < a.F; f += 32) s += __ldcg(a.llf + f);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) a.trace[a.trace_slot] = s;
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

// FP64 fixed-point update of P(f) (Eq. FPI, K sweeps) from the finalised
// V_i in shared memory.  Lane 0 inverts P, lanes i < I solve column i.
template <int I>
__device__ void p_update(const FastArgs& a, int f, const double* sV, double (*sPn)[I][2],
                         double (*sQ)[I][2], int* sbad) {
  const int lane = threadIdx.x & 31;  // called by one full warp
  if (lane == 0) *sbad = 0;
  if (lane < I * I) {
    sPn[lane / I][lane % I][0] = a.P[((size_t)f * I * I + lane) * 2];
    sPn[lane / I][lane % I][1] = a.P[((size_t)f * I * I + lane) * 2 + 1];
  }
  __syncwarp();
  for (int sweep = 0; sweep < a.K; ++sweep) {
    if (lane == 0) {
      cpx<double> A[I][I];
#pragma unroll
      for (int r = 0; r < I; ++r)
#pragma unroll
        for (int c = 0; c < I; ++c) A[r][c] = mk(sPn[r][c][0], sPn[r][c][1]);
      double ld2;
      if (!gj_inverse<I>(A, ld2)) *sbad = 1;
      // Q = (P^{-1})^H: Q[r][c] = conj(Pinv[c][r])
#pragma unroll
      for (int r = 0; r < I; ++r)
#pragma unroll
        for (int c = 0; c < I; ++c) {
          sQ[r][c][0] = A[c][r].re;
          sQ[r][c][1] = -A[c][r].im;
        }
    }
    __syncwarp();
    if (lane < I) {
      const int i = lane;
      cpx<double> V[I][I], b[I], x[I];
      unpack_herm<I>(sV + i * I * I, V);
#pragma unroll
      for (int r = 0; r < I; ++r) b[r] = mk(sQ[r][i][0], sQ[r][i][1]);
      if (!chol_solve<I>(V, b, x)) *sbad = 1;
#pragma unroll
      for (int r = 0; r < I; ++r) {
        sPn[r][i][0] = x[r].re;
        sPn[r][i][1] = x[r].im;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    cpx<double> A[I][I];
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) A[r][c] = mk(sPn[r][c][0], sPn[r][c][1]);
    double ld2 = 0.0;
    if (!gj_inverse<I>(A, ld2)) *sbad = 1;
    a.logdet[f] = ld2;
    atomicAdd(a.ops, (unsigned long long)(I + 1) * a.K);
    if (*sbad) raise_status(a.status, kDevSingular, f);
  }
  __syncwarp();
  if (lane < I * I) {
    a.P[((size_t)f * I * I + lane) * 2] = sPn[lane / I][lane % I][0];
    a.P[((size_t)f * I * I + lane) * 2 + 1] = sPn[lane / I][lane % I][1];
  }
}

// -------------------------------------------------------------- P solve
// One warp per frequency: sum pass B's slots into V_i (FP64, slot order),
// then the fixed-point update of P(f) and ln|det P(f)|^2.
constexpr int kSolveWarps = 4;

template <int I>
__global__ void __launch_bounds__(32 * kSolveWarps) k_psolve(FastArgs a) {
  constexpr int NV = I * I * I;
  __shared__ double sV[kSolveWarps][NV];
  __shared__ double sPn[kSolveWarps][I][I][2];
  __shared__ double sQ[kSolveWarps][I][I][2];
  __shared__ int sbad[kSolveWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kSolveWarps + warp;
  if (f >= a.F) return;  // whole warps only
  const Partition pt = a.part;
  const int ns = pt.nslots(f);
  for (int t = lane; t < NV; t += 32) {
    const double s = sum_slots(a.part_buf, f, ns, pt.max_slots, NV, t) / a.N;
    if (!isfinite(s)) raise_status(a.status, kDevNonfinite, f);
    sV[warp][t] = s;
  }
  __syncwarp();
  p_update<I>(a, f, sV[warp], sPn[warp], sQ[warp], &sbad[warp]);
}

// -------------------------------------------------------------- prep
// Per frequency (one thread each): ln|det P|^2 and P^{-H} of the current P.
template <int I>
__global__ void k_prep(FastArgs a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.F) return;
  cpx<double> A[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c)
      A[r][c] = mk(a.P[((size_t)f * I * I + r * I + c) * 2], a.P[((size_t)f * I * I + r * I + c) * 2 + 1]);
  double ld2 = 0.0;
  if (!gj_inverse<I>(A, ld2)) raise_status(a.status, kDevSingular, f);
  a.logdet[f] = ld2;
  if (a.pinvH) {
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) {  // (P^{-1})^H [r][c] = conj(Pinv[c][r])
        a.pinvH[((size_t)f * I * I + r * I + c) * 2] = A[c][r].re;
        a.pinvH[((size_t)f * I * I + r * I + c) * 2 + 1] = -A[c][r].im;
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
  const long long total = (long long)pt.F * pt.Uf;
  const long long u0 = (long long)blockIdx.x * pt.upb;
  const long long u1 = min(u0 + pt.upb, total);
  const long long row = a.ld / FU;
  const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y);
  const VV* __restrict__ v = reinterpret_cast<const VV*>(a.v);
  VY* __restrict__ out = reinterpret_cast<VY*>(a.out);

  for (long long u = u0; u < u1;) {
    const int f = (int)(u / pt.Uf);
    const int k0 = (int)(u - (long long)f * pt.Uf);
    const int k1 = (int)min((long long)pt.Uf, k0 + (u1 - u));
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
      for (int m = 0; m < I; ++m) yu[m] = y[((size_t)m * pt.F + f) * row + k];
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = v[((size_t)j * pt.F + f) * row + k];
      VY o[J][I];
#pragma unroll
      for (int e = 0; e < FU; ++e) {
        const bool valid = k * FU + e < a.N;
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
        for (int r = 0; r < I; ++r) out[(((size_t)j * I + r) * pt.F + f) * row + k] = o[j][r];
    }
    u += k1 - k0;
  }
}

}  // namespace ffca
