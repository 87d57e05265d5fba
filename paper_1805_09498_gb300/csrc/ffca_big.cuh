// Per-problem FP64 kernels for arrays of more than four microphones
// (I > 4), where the cofactor forms of the small kernels would take too many
// operations: the same lane layout (lane (g, i) owns column i of problem g,
// 32 / I problems per warp), with each lane's I x I matrices in its own slice
// of shared memory (padded by one element so that the lanes' 16-byte
// accesses fall in distinct banks).
//
//   k_psolve_big  Eq. FPI: [P^{-H}]_i by Gaussian elimination with partial
//                 pivoting of P^H x = e_i, then p_i = V_i^{-1} [P^{-H}]_i by
//                 Cholesky (V_i Hermitian positive definite), K sweeps, all
//                 columns from one P^{-H} per sweep; ln|det P|^2 of the new P
//                 from the pivots of its elimination.
//   k_prep_big    ln|det P|^2, the pass-A table and, if asked, P^{-H}.
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

template <int I>
struct BigLane {
  static constexpr int LD = I * I + 1;  // complex elements per lane slice (padded)
  static constexpr int SLICES = 2;      // elimination matrix, Cholesky factor
  static constexpr int G = 32 / I;      // problems per warp
  // per block (one warp): the lanes' slices and each problem's new P
  static constexpr int SMEM = (32 * SLICES * LD + G * I * I) * (int)sizeof(cpx<double>);
};

__device__ inline cpx<double> crecip(cpx<double> a) {
  const double r = 1.0 / cabs2(a);
  return mk(a.re * r, -a.im * r);
}

// LU with partial pivoting of the I x I matrix A (row-major, in place) and,
// if b != nullptr, the solution of A x = b in place of b.  Returns
// sum_k ln|u_kk|^2 = ln|det A|^2 (-inf for a zero pivot).
template <int I>
__device__ double gauss_solve(cpx<double>* A, cpx<double>* b) {
  double lg = 0.0;
  for (int k = 0; k < I; ++k) {
    int p = k;
    double best = cabs2(A[k * I + k]);
    for (int r = k + 1; r < I; ++r) {
      const double m = cabs2(A[r * I + k]);
      if (m > best) {
        best = m;
        p = r;
      }
    }
    if (!(best > 0.0)) return -INFINITY;
    if (p != k) {
      for (int c = k; c < I; ++c) {
        const cpx<double> t = A[k * I + c];
        A[k * I + c] = A[p * I + c];
        A[p * I + c] = t;
      }
      if (b) {
        const cpx<double> t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
    lg += log(best);
    const cpx<double> inv = crecip(A[k * I + k]);
    for (int r = k + 1; r < I; ++r) {
      const cpx<double> m = cmul(A[r * I + k], inv);
      for (int c = k + 1; c < I; ++c) A[r * I + c] = csub(A[r * I + c], cmul(m, A[k * I + c]));
      if (b) b[r] = csub(b[r], cmul(m, b[k]));
    }
  }
  if (b) {
    for (int k = I - 1; k >= 0; --k) {
      cpx<double> s = b[k];
      for (int c = k + 1; c < I; ++c) s = csub(s, cmul(A[k * I + c], b[c]));
      b[k] = cmul(s, crecip(A[k * I + k]));
    }
  }
  return lg;
}

// Cholesky V = L L^H in place (lower triangle, row-major); false if a pivot
// is at or below kCholRtol times its diagonal entry (rank deficient).
template <int I>
__device__ bool cholesky(cpx<double>* V) {
  for (int k = 0; k < I; ++k) {
    double d = V[k * I + k].re;
    const double d0 = d;
    for (int c = 0; c < k; ++c) d -= cabs2(V[k * I + c]);
    if (!(d > kCholRtol * d0) || !isfinite(d)) return false;
    const double lkk = sqrt(d);
    V[k * I + k] = mk(lkk, 0.0);
    const double rl = 1.0 / lkk;
    for (int r = k + 1; r < I; ++r) {
      cpx<double> s = V[r * I + k];
      for (int c = 0; c < k; ++c) s = csub(s, cmul(V[r * I + c], cconj(V[k * I + c])));
      V[r * I + k] = cscale(s, rl);
    }
  }
  return true;
}

// x <- (L L^H)^{-1} x with the factor from cholesky().
template <int I>
__device__ void chol_solve(const cpx<double>* L, cpx<double>* x) {
  for (int k = 0; k < I; ++k) {  // L z = x
    cpx<double> s = x[k];
    for (int c = 0; c < k; ++c) s = csub(s, cmul(L[k * I + c], x[c]));
    x[k] = cscale(s, 1.0 / L[k * I + k].re);
  }
  for (int k = I - 1; k >= 0; --k) {  // L^H p = z
    cpx<double> s = x[k];
    for (int r = k + 1; r < I; ++r) s = csub(s, cmul(cconj(L[r * I + k]), x[r]));
    x[k] = cscale(s, 1.0 / L[k * I + k].re);
  }
}

template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_psolve_big(FastArgs a) {
  using BL = BigLane<I>;
  constexpr int G = BL::G;
  constexpr int NV = I * I * I;
  extern __shared__ __align__(16) unsigned char big_smem[];
  cpx<double>* lanes = reinterpret_cast<cpx<double>*>(big_smem);
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f0 = blockIdx.x * G + g;
  const bool active = g < G && f0 < a.F;
  const int f = active ? f0 : 0;  // idle lanes shadow problem 0 and write nothing
  cpx<double>* E = lanes + (size_t)lane * BL::SLICES * BL::LD;  // elimination matrix
  cpx<double>* Lc = E + BL::LD;                                  // Cholesky factor of V_i
  cpx<double>* Pn = lanes + (size_t)32 * BL::SLICES * BL::LD + (size_t)(g < G ? g : 0) * I * I;  // new P
  const Partition pt = a.part;

  if (active && a.lam_next) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
    for (int j = 0; j < J; ++j) {
      const double l = a.lam_next[(size_t)f * J * I + j * I + i];
      a.lam[(size_t)f * J * I + j * I + i] = l;
      ta->lam[j][i] = (T)l;
    }
  }
  // V_i from the slots (packed Hermitian: diagonal, then (re, im) above it)
  {
    const int ns = pt.nslots(f);
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV + i * I * I;
    const double sc = pt.inv_n(f);
    auto slot_sum = [&](int m) {
      double s = 0.0;
      for (int k = 0; k < ns; ++k) s += __ldcg(base + (size_t)k * NV + m);
      return s * sc;
    };
    int m = I;
    for (int r = 0; r < I; ++r) {
      Lc[r * I + r] = mk(slot_sum(r), 0.0);
      for (int c = r + 1; c < I; ++c) {
        const cpx<double> z = mk(slot_sum(m), slot_sum(m + 1));
        Lc[r * I + c] = z;
        Lc[c * I + r] = cconj(z);
        m += 2;
      }
    }
  }
  bool bad = false;
  for (int r = 0; r < I * I; ++r) bad |= !isfinite(Lc[r].re) || !isfinite(Lc[r].im);
  if (active && bad) raise_status(a.status, kDevNonfinite, f);
  bool singular = !cholesky<I>(Lc);

  // current P of the problem, gathered in shared memory (lane (g, c) loads column c)
  for (int r = 0; r < I; ++r)
    Pn[r * I + i] = mk(a.P[((size_t)f * I * I + r * I + i) * 2], a.P[((size_t)f * I * I + r * I + i) * 2 + 1]);
  __syncwarp();
  cpx<double> x[I];
  for (int sweep = 0; sweep < a.K; ++sweep) {
    // [P^{-H}]_i: solve P^H x = e_i
    for (int r = 0; r < I; ++r)
      for (int c = 0; c < I; ++c) E[r * I + c] = cconj(Pn[c * I + r]);
    for (int r = 0; r < I; ++r) x[r] = mk(r == i ? 1.0 : 0.0, 0.0);
    double lg;
    {
      cpx<double> b[I];
      for (int r = 0; r < I; ++r) b[r] = x[r];
      lg = gauss_solve<I>(E, b);
      for (int r = 0; r < I; ++r) x[r] = b[r];
    }
    singular |= !isfinite(lg);
    if (!singular) chol_solve<I>(Lc, x);  // p_i = V_i^{-1} [P^{-H}]_i
    __syncwarp();                         // every lane of the problem has read the old P
    for (int r = 0; r < I; ++r) Pn[r * I + i] = x[r];
    __syncwarp();
  }
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
    for (int r = 0; r < I; ++r) {
      const cpx<double> pr = Pn[r * I + i];
      a.P[((size_t)f * I * I + r * I + i) * 2] = pr.re;
      a.P[((size_t)f * I * I + r * I + i) * 2 + 1] = pr.im;
      ta->pre[r][i] = (T)pr.re;
      ta->pim[r][i] = (T)pr.im;
    }
    if (singular) raise_status(a.status, kDevSingular, f);
    if (i == 0) {
      atomicAdd(a.ops, (unsigned long long)(I + 1) * a.K);
      for (int r = 0; r < I * I; ++r) E[r] = Pn[r];
      const double lg = gauss_solve<I>(E, nullptr);
      if (!isfinite(lg)) raise_status(a.status, kDevSingular, f);
      a.logdet[f] = lg;
    }
  }
  if (a.trace) {
    unsigned last = 0;
    if (lane == 0) {
      last = atomicAdd(a.gcnt, 1u) == gridDim.x - 1;
      if (last) *a.gcnt = 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      finalize_trace(a);
    }
  }
}

template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_prep_big(FastArgs a) {
  using BL = BigLane<I>;
  constexpr int G = BL::G;
  extern __shared__ __align__(16) unsigned char big_smem[];
  cpx<double>* lanes = reinterpret_cast<cpx<double>*>(big_smem);
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f = blockIdx.x * G + g;
  if (g >= G || f >= a.F) return;
  cpx<double>* E = lanes + (size_t)lane * BL::SLICES * BL::LD;
  ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
  for (int r = 0; r < I; ++r) {
    ta->pre[r][i] = (T)a.P[((size_t)f * I * I + r * I + i) * 2];
    ta->pim[r][i] = (T)a.P[((size_t)f * I * I + r * I + i) * 2 + 1];
  }
  for (int j = 0; j < J; ++j) ta->lam[j][i] = (T)a.lam[(size_t)f * J * I + j * I + i];
  // P^H in the lane's slice; column i of P^{-H} solves P^H x = e_i
  for (int r = 0; r < I; ++r)
    for (int c = 0; c < I; ++c)
      E[r * I + c] = mk(a.P[((size_t)f * I * I + c * I + r) * 2], -a.P[((size_t)f * I * I + c * I + r) * 2 + 1]);
  cpx<double> b[I];
  for (int r = 0; r < I; ++r) b[r] = mk(r == i ? 1.0 : 0.0, 0.0);
  const double lg = gauss_solve<I>(E, b);  // ln|det P^H|^2 = ln|det P|^2
  if (!isfinite(lg)) raise_status(a.status, kDevSingular, f);
  if (i == 0) a.logdet[f] = lg;
  if (a.pinvH) {
    for (int r = 0; r < I; ++r) {
      a.pinvH[((size_t)f * I * I + r * I + i) * 2] = b[r].re;
      a.pinvH[((size_t)f * I * I + r * I + i) * 2 + 1] = b[r].im;
    }
  }
}

// Wiener filter for I > 4 (Eq. MMSE0): P, P^{-H} and Lambda of the frequency
// in shared memory in the per-point precision; each thread forms y~ and
// 1/sigma for its unit's frames once, then each source's output in turn.
template <typename T, int I, int J>
__global__ void __launch_bounds__(kBlock) k_wiener_big(FastArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  constexpr int FU = Vec<T>::FU;
  __shared__ cpx<T> sP[I][I], sQ[I][I];
  __shared__ T sLam[J][I];

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
    for (int t = threadIdx.x; t < I * I; t += kBlock) {
      const int r = t / I, c = t % I;
      sP[r][c] = mk<T>((T)a.P[((size_t)f * I * I + t) * 2], (T)a.P[((size_t)f * I * I + t) * 2 + 1]);
      sQ[r][c] = mk<T>((T)a.pinvH[((size_t)f * I * I + t) * 2], (T)a.pinvH[((size_t)f * I * I + t) * 2 + 1]);
    }
    for (int t = threadIdx.x; t < J * I; t += kBlock) sLam[t / I][t % I] = (T)a.lam[(size_t)f * J * I + t];
    __syncthreads();
    for (int k = k0 + threadIdx.x; k < k1; k += kBlock) {
      cpx<T> yt[FU][I];
      T rs[FU][I];
      VV vu[J];
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = v[((size_t)j * pt.F + f) * row + k];
      {
        VY yu[I];
#pragma unroll
        for (int m = 0; m < I; ++m) yu[m] = y[((size_t)m * pt.F + f) * row + k];
#pragma unroll
        for (int e = 0; e < FU; ++e) {
#pragma unroll
          for (int i = 0; i < I; ++i) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int m = 0; m < I; ++m) cfmac(s, sP[m][i], yframe(yu[m], e));
            yt[e][i] = s;
            T sg = vframe(vu[0], e) * sLam[0][i];
#pragma unroll
            for (int j = 1; j < J; ++j) sg = fma(vframe(vu[j], e), sLam[j][i], sg);
            rs[e][i] = recip(sg);
          }
        }
      }
#pragma unroll 1
      for (int j = 0; j < J; ++j) {
        VY o[I];
#pragma unroll
        for (int e = 0; e < FU; ++e) {
          const bool valid = k * FU + e < a.N;
          cpx<T> z[I];
#pragma unroll
          for (int i = 0; i < I; ++i) z[i] = cscale(yt[e][i], vframe(vu[j], e) * sLam[j][i] * rs[e][i]);
#pragma unroll
          for (int r = 0; r < I; ++r) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int i = 0; i < I; ++i) cfma(s, sQ[r][i], z[i]);
            yset(o[r], e, valid ? s : mk<T>(0, 0));
          }
        }
#pragma unroll
        for (int r = 0; r < I; ++r) out[(((size_t)j * I + r) * pt.F + f) * row + k] = o[r];
      }
    }
    u += k1 - k0;
  }
}

}  // namespace ffca
