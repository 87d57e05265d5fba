// Conventional FCA (full-rank spatial covariance analysis), the EM algorithm
// of Sec. 3.3, as the in-repo GPU baseline.  Per time-frequency point it
// builds R = sum_j v_j S_j, inverts it (a full I x I Hermitian inverse), and
// forms the products R_j R^{-1} and R_j R^{-1} R_j of Eqs. MMSE and
// postquadexp: the per-point inversions and multiplications that Sec. 3.4
// counts and that FastFCA-AS removes.
//
//   k_fca_prep   per frequency (FP64): S_j^{-1} by cofactors, and the table of
//                S_j, S_j^{-1} in the per-point precision.
//   k_fca_em     per point: E-step, v_j <- (1/I) tr(S_j^{-1} (mu_j mu_j^H + Phi_j))
//                in place (Eq. vupdate, current S_j), partial sums over n of
//                (mu_j mu_j^H + Phi_j) / v_j^new (Eq. Supdate) and of the terms
//                of Eq. L1 (ln det R + y^H R^{-1} y), into per-frequency slots.
//   k_fca_final  per frequency (FP64): S_j from the slots, S_j^{-1}, the table,
//                the frequency's log-likelihood; the last warp sums the trace.
// Layouts: y [I][F][ld], v [J][F][ld] as for FastFCA-AS; S [F][J][I][I]
// complex128 row-major (Hermitian positive definite).
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

struct FcaArgs {
  Partition part;
  int F, N, ld;
  const void* y;
  void* v;
  double* S;               // [F][J][I][I] complex, in/out
  void* tab;               // [F] FcaParams in the per-point precision
  double* part_buf;        // [F][max_slots][NV]
  double* llf;             // [F]
  double* trace;           // [kTraceCap]
  int trace_slot;
  unsigned* gcnt;
  unsigned* status;
  unsigned long long* ops;    // matrix inversions, counted as in Sec. 3.4
  unsigned long long* mults;  // matrix-matrix multiplications, counted as in Sec. 3.4
  double inv_n;
};

// S_j(f) and S_j(f)^{-1}, interleaved complex, in the per-point precision.
template <typename T, int I, int J>
struct FcaParams {
  T s[J][I][I][2];
  T sinv[J][I][I][2];
  static constexpr int BYTES = (int)(sizeof(T) * 4 * J * I * I);
};
template <typename T, int I, int J>
__device__ inline FcaParams<T, I, J>* fca_tab(const FcaArgs& a, int f) {
  return reinterpret_cast<FcaParams<T, I, J>*>(static_cast<char*>(a.tab) + (size_t)f * FcaParams<T, I, J>::BYTES);
}

// Complex I x I helpers in the per-point precision.
template <typename T, int I>
__device__ inline cpx<T> minor3(const cpx<T> (&A)[I][I], int r, int c) {
  if constexpr (I == 1) {
    return mk<T>(1, 0);
  } else {
    int rows[I - 1], cols[I - 1];
#pragma unroll
    for (int k = 0, nr = 0, nc = 0; k < I; ++k) {
      if (k != r) rows[nr++] = k;
      if (k != c) cols[nc++] = k;
    }
    if constexpr (I == 2) {
      return A[rows[0]][cols[0]];
    } else if constexpr (I == 3) {
      return csub(cmul(A[rows[0]][cols[0]], A[rows[1]][cols[1]]), cmul(A[rows[0]][cols[1]], A[rows[1]][cols[0]]));
    } else {
      auto e = [&](int rr, int cc) { return A[rows[rr]][cols[cc]]; };
      cpx<T> d = cmul(e(0, 0), csub(cmul(e(1, 1), e(2, 2)), cmul(e(1, 2), e(2, 1))));
      d = csub(d, cmul(e(0, 1), csub(cmul(e(1, 0), e(2, 2)), cmul(e(1, 2), e(2, 0)))));
      return cadd(d, cmul(e(0, 2), csub(cmul(e(1, 0), e(2, 1)), cmul(e(1, 1), e(2, 0)))));
    }
  }
}

// Inverse of a Hermitian positive definite I x I matrix by cofactors
// (A^{-1} = C^T / det A); returns det A (real and positive for HPD A).
template <typename T, int I>
__device__ inline T herm_inverse(const cpx<T> (&A)[I][I], cpx<T> (&Ainv)[I][I]) {
  cpx<T> C[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) {
      const cpx<T> m = minor3<T, I>(A, r, c);
      C[r][c] = ((r + c) & 1) ? mk<T>(-m.re, -m.im) : m;
    }
  T det = (T)0;
#pragma unroll
  for (int c = 0; c < I; ++c) det += A[0][c].re * C[0][c].re - A[0][c].im * C[0][c].im;
  const T rd = recip(det);
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) Ainv[r][c] = cscale(C[c][r], rd);
  return det;
}

// -------------------------------------------------------------- prep (FP64)
// One thread per frequency: S_j^{-1} by cofactors and the per-point table.
template <typename T, int I, int J>
__global__ void k_fca_prep(FcaArgs a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.F) return;
  FcaParams<T, I, J>* tp = fca_tab<T, I, J>(a, f);
  for (int j = 0; j < J; ++j) {
    cpx<double> S[I][I], Si[I][I];
    const double* sp = a.S + ((size_t)(f * J + j) * I * I) * 2;
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) S[r][c] = mk(sp[(r * I + c) * 2], sp[(r * I + c) * 2 + 1]);
    const double det = herm_inverse<double, I>(S, Si);
    if (!(det > 0.0) || !isfinite(det)) raise_status(a.status, kDevSingular, f);
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) {
        tp->s[j][r][c][0] = (T)S[r][c].re;
        tp->s[j][r][c][1] = (T)S[r][c].im;
        tp->sinv[j][r][c][0] = (T)Si[r][c].re;
        tp->sinv[j][r][c][1] = (T)Si[r][c].im;
      }
  }
}

// -------------------------------------------------------------- EM pass
template <typename T, int I, int J, bool UPDATE>
__global__ void __launch_bounds__(kBlock) k_fca_em(FcaArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  constexpr int FU = Vec<T>::FU;
  constexpr int I2 = I * I;
  constexpr int NS = UPDATE ? J * I2 : 0;  // packed Hermitian (mu mu^H + Phi) / v_new per j
  constexpr int NV = NS + 1;               // then ln det R + y^H R^{-1} y
  using Red = ButterflyReduce<T, NV, kWarps, false>;
  __shared__ typename Red::Smem red;
  __shared__ FcaParams<T, I, J> sp;

  const Partition pt = a.part;
  const long long total = (long long)pt.F * pt.Uf;
  const long long u0 = (long long)blockIdx.x * pt.upb;
  const long long u1 = min(u0 + pt.upb, total);
  const long long row = a.ld / FU;
  const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y);
  VV* __restrict__ v = reinterpret_cast<VV*>(a.v);

  for (long long u = u0; u < u1;) {
    const int f = (int)(u / pt.Uf);
    const int k0 = (int)(u - (long long)f * pt.Uf);
    const int k1 = (int)min((long long)pt.Uf, k0 + (u1 - u));
    __syncthreads();  // the previous segment is done with sp
    {
      const T* src = reinterpret_cast<const T*>(fca_tab<T, I, J>(a, f));
      T* dst = reinterpret_cast<T*>(&sp);
      for (int t = threadIdx.x; t < FcaParams<T, I, J>::BYTES / (int)sizeof(T); t += kBlock) dst[t] = src[t];
    }
    __syncthreads();
    T acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = (T)0;

    for (int k = k0 + threadIdx.x; k < k1; k += kBlock) {
      VY yu[I];
      VV vu[J];
#pragma unroll
      for (int m = 0; m < I; ++m) yu[m] = y[((size_t)m * pt.F + f) * row + k];
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = v[((size_t)j * pt.F + f) * row + k];
#pragma unroll
      for (int e = 0; e < FU; ++e) {
        if (k * FU + e >= a.N) continue;
        cpx<T> yv[I];
#pragma unroll
        for (int m = 0; m < I; ++m) yv[m] = yframe(yu[m], e);
        // R = sum_j v_j S_j and its inverse (Eq. L1's covariance)
        cpx<T> R[I][I], Ri[I][I];
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = 0; c < I; ++c) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int j = 0; j < J; ++j) {
              const T vj = vframe(vu[j], e);
              s.re = fma(vj, sp.s[j][r][c][0], s.re);
              s.im = fma(vj, sp.s[j][r][c][1], s.im);
            }
            R[r][c] = s;
          }
        const T detR = herm_inverse<T, I>(R, Ri);
        // z = R^{-1} y, y^H R^{-1} y
        cpx<T> z[I];
        T quad = (T)0;
#pragma unroll
        for (int r = 0; r < I; ++r) {
          cpx<T> s = mk<T>(0, 0);
#pragma unroll
          for (int c = 0; c < I; ++c) cfma(s, Ri[r][c], yv[c]);
          z[r] = s;
        }
#pragma unroll
        for (int r = 0; r < I; ++r) quad += yv[r].re * z[r].re + yv[r].im * z[r].im;
        acc[NS] += logx(detR) + quad;
        if constexpr (UPDATE) {
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const T vj = vframe(vu[j], e);
            // G = R_j R^{-1} (Eq. MMSE), mu_j = G y, Phi_j = R_j - G R_j (Eq. postquadexp)
            cpx<T> G[I][I];
#pragma unroll
            for (int r = 0; r < I; ++r)
#pragma unroll
              for (int c = 0; c < I; ++c) {
                cpx<T> s = mk<T>(0, 0);
#pragma unroll
                for (int q = 0; q < I; ++q) cfma(s, mk<T>(vj * sp.s[j][r][q][0], vj * sp.s[j][r][q][1]), Ri[q][c]);
                G[r][c] = s;
              }
            cpx<T> mu[I];
#pragma unroll
            for (int r = 0; r < I; ++r) {
              cpx<T> s = mk<T>(0, 0);
#pragma unroll
              for (int c = 0; c < I; ++c) cfma(s, G[r][c], yv[c]);
              mu[r] = s;
            }
            cpx<T> Cm[I][I];  // mu mu^H + Phi
#pragma unroll
            for (int r = 0; r < I; ++r)
#pragma unroll
              for (int c = 0; c < I; ++c) {
                cpx<T> s = mk<T>(vj * sp.s[j][r][c][0], vj * sp.s[j][r][c][1]);  // R_j
#pragma unroll
                for (int q = 0; q < I; ++q) {
                  const cpx<T> Rqc = mk<T>(vj * sp.s[j][q][c][0], vj * sp.s[j][q][c][1]);
                  const cpx<T> g = cmul(G[r][q], Rqc);
                  s.re -= g.re;
                  s.im -= g.im;
                }
                cfma(s, mu[r], cconj(mu[c]));
                Cm[r][c] = s;
              }
            // Eq. vupdate with the current S_j^{-1}: tr(S_j^{-1} C) = sum_rc Sinv_rc C_cr
            T tr = (T)0;
#pragma unroll
            for (int r = 0; r < I; ++r)
#pragma unroll
              for (int c = 0; c < I; ++c)
                tr += sp.sinv[j][r][c][0] * Cm[c][r].re - sp.sinv[j][r][c][1] * Cm[c][r].im;
            const T vn = tr * (T)(1.0 / I);
            vset(vu[j], e, vn);
            const T rv = recip(vn);
            // Eq. Supdate numerator, packed Hermitian: diagonal, then (re, im) above it
            int m = I;
#pragma unroll
            for (int r = 0; r < I; ++r) {
              acc[j * I2 + r] = fma(Cm[r][r].re, rv, acc[j * I2 + r]);
#pragma unroll
              for (int c = r + 1; c < I; ++c) {
                acc[j * I2 + m] = fma(Cm[r][c].re, rv, acc[j * I2 + m]);
                acc[j * I2 + m + 1] = fma(Cm[r][c].im, rv, acc[j * I2 + m + 1]);
                m += 2;
              }
            }
          }
        }
      }
      if constexpr (UPDATE) {
#pragma unroll
        for (int j = 0; j < J; ++j) v[((size_t)j * pt.F + f) * row + k] = vu[j];
      }
    }
    T lo[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) lo[q] = (T)0;
    const int slot = (int)blockIdx.x - pt.first_block(f);
    Red::run(acc, lo, red, a.part_buf + ((size_t)f * pt.max_slots + slot) * NV);
    if (UPDATE && threadIdx.x == 0) {
      // per point: one inversion of R (Eqs. MMSE, postquadexp) and, per j, the
      // products R_j R^{-1} and (R_j R^{-1}) R_j
      const long long n1 = min((long long)k1 * FU, (long long)a.N) - (long long)k0 * FU;
      if (n1 > 0) {
        atomicAdd(a.ops, (unsigned long long)n1);
        atomicAdd(a.mults, (unsigned long long)(2 * J) * n1);
      }
    }
    u += k1 - k0;
  }
}

// -------------------------------------------------------------- finalise (FP64)
// One thread per frequency: S_j = (1/N) sum_n (mu mu^H + Phi) / v_j (Eq.
// Supdate) from the slots, S_j^{-1} (cofactors), the table, and the
// frequency's log-likelihood of the entering state (Eq. L1); the last block
// sums the trace.  With UPDATE false only the log-likelihood.
template <typename T, int I, int J, bool UPDATE>
__global__ void k_fca_final(FcaArgs a) {
  constexpr int I2 = I * I;
  constexpr int NS = UPDATE ? J * I2 : 0;
  constexpr int NV = NS + 1;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < a.F) {
    const Partition pt = a.part;
    const int ns = pt.nslots(f);
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV;
    double lsum = 0.0;
    for (int k = 0; k < ns; ++k) lsum += __ldcg(base + (size_t)k * NV + NS);
    const double lf = -(double)I * a.N * kLnPi - lsum;
    if (!isfinite(lf)) raise_status(a.status, kDevNonfinite, f);
    a.llf[f] = lf;
    if constexpr (UPDATE) {
      FcaParams<T, I, J>* tp = fca_tab<T, I, J>(a, f);
      for (int j = 0; j < J; ++j) {
        double pk[I2];
#pragma unroll
        for (int m = 0; m < I2; ++m) pk[m] = 0.0;
        for (int k = 0; k < ns; ++k)
#pragma unroll
          for (int m = 0; m < I2; ++m) pk[m] += __ldcg(base + (size_t)k * NV + j * I2 + m);
#pragma unroll
        for (int m = 0; m < I2; ++m) pk[m] *= a.inv_n;
        cpx<double> S[I][I], Si[I][I];
        unpack_herm<I>(pk, S);
        const double det = herm_inverse<double, I>(S, Si);
        if (!(det > 0.0) || !isfinite(det)) raise_status(a.status, kDevSingular, f);
        double* sp = a.S + ((size_t)(f * J + j) * I * I) * 2;
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = 0; c < I; ++c) {
            sp[(r * I + c) * 2] = S[r][c].re;
            sp[(r * I + c) * 2 + 1] = S[r][c].im;
            tp->s[j][r][c][0] = (T)S[r][c].re;
            tp->s[j][r][c][1] = (T)S[r][c].im;
            tp->sinv[j][r][c][0] = (T)Si[r][c].re;
            tp->sinv[j][r][c][1] = (T)Si[r][c].im;
          }
      }
      atomicAdd(a.ops, (unsigned long long)J);  // S_j^{-1}: J inversions per frequency
    }
    __threadfence();
  }
  __syncthreads();
  __shared__ int last;
  if (threadIdx.x == 0) {
    last = atomicAdd(a.gcnt, 1u) == gridDim.x - 1;
    if (last) *a.gcnt = 0u;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    const int lane = threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f2 = lane; f2 < a.F; f2 += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (f2 + 32 * u < a.F) s[u] += __ldcg(a.llf + f2 + 32 * u);
    }
    double t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) a.trace[a.trace_slot] = t;
  }
}

}  // namespace ffca
