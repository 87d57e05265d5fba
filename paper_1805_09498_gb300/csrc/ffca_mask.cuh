// Mask-based initialisation of (v, Lambda, P) from caller-given
// time-frequency masks (Sec. 5 initialises the parameters by mask-based
// covariance matrix estimation; the masking method itself is not part of
// this library).  Readings of the steps the paper does not state:
//
//   k_mask_cov  R_j(f) = sum_n m_j(n,f) y y^H / sum_n m_j(n,f), one CTA per
//               (problem, source), sums over the frames in FP64.
//   k_mask_ajd  per problem (one thread, FP64): P from the generalized
//               eigenvectors of (R_1, R_y), R_y = sum_j R_j (the GEVD that
//               gives P and Lambda for two sources, Sec. 4.1): R_y = L L^H,
//               W = L^{-1} R_1 L^{-H} = U diag(w) U^H by cyclic Jacobi
//               rotations, ascending w, P = L^{-H} U with each column turned
//               in phase so that its entry of largest magnitude is real and
//               positive; then `sweeps` alternations lambda_ji = p_i^H R_j p_i,
//               p_i <- V_i^{-1} [P^{-H}]_i with V_i = (1/J) sum_j R_j / lambda_ji
//               (Eq. FPI on the covariances); finally lambda_ji = p_i^H R_j p_i.
//   k_mask_v    v_j(n,f) = max(m_j(n,f), delta) (1/I) sum_i |y~_i|^2 / lambda_ji,
//               y~ = P^H y (the masked image's quadratic form under S_j).
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

constexpr int kMaskMaxJ = 6;

struct MaskArgs {
  Partition part;    // problems: frames, rows and offsets (pass A's partition)
  int I, J, ld;
  const void* y;     // the mixture (layout of the context)
  const void* m;     // masks, layout of v, the precision's real type
  void* v;           // out: source powers
  double* lam;       // out: [problems][J][I]
  double* P;         // out: [problems][I][I] complex
  double* R;         // workspace: [problems][J][I][I] complex, the masked covariances
  int sweeps;
  double delta;
  unsigned* status;
};

// ------------------------------------------------------------ covariances
template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_mask_cov(MaskArgs a) {
  using C = cpx<T>;
  constexpr int NV = I * I + 1;  // the packed Hermitian sum (diagonal, (re, im) above it), then sum m
  __shared__ typename BlockReduce<double, NV>::Smem red;
  __shared__ double tot[NV];
  const int p = blockIdx.x, j = blockIdx.y;
  const Partition& pt = a.part;
  const int n = pt.frames(p);
  const long long rlen = pt.row_len(p, a.ld), off = pt.frame_off(p), fr = pt.freq(p);
  const C* y = reinterpret_cast<const C*>(a.y) + (size_t)a.I * pt.Fm * off + fr * rlen;
  const T* m = reinterpret_cast<const T*>(a.m) + (size_t)a.J * pt.Fm * off + ((long long)j * pt.Fm + fr) * rlen;
  const size_t rs = (size_t)pt.Fm * rlen;  // stride between the problem's rows
  double hi[NV], lo[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) hi[q] = lo[q] = 0.0;
  for (int t = threadIdx.x; t < n; t += kBlock) {
    const double w = (double)m[t];
    cpx<double> z[I];
#pragma unroll
    for (int r = 0; r < I; ++r) {
      const C c = y[r * rs + t];
      z[r] = mk((double)c.re, (double)c.im);
    }
    int q = I;
#pragma unroll
    for (int r = 0; r < I; ++r) {
      hi[r] = fma(w, cabs2(z[r]), hi[r]);
#pragma unroll
      for (int c = r + 1; c < I; ++c) {  // z_r conj(z_c)
        hi[q] = fma(w, z[r].re * z[c].re + z[r].im * z[c].im, hi[q]);
        hi[q + 1] = fma(w, z[r].im * z[c].re - z[r].re * z[c].im, hi[q + 1]);
        q += 2;
      }
    }
    hi[NV - 1] += w;
  }
  BlockReduce<double, NV>::run(hi, lo, red, tot);
  __syncthreads();
  const double ws = tot[NV - 1];
  if (threadIdx.x == 0 && !(ws > 0.0)) raise_status(a.status, kDevNonfinite, p);
  double* R = a.R + ((size_t)p * a.J + j) * I * I * 2;
  for (int e = threadIdx.x; e < I * I; e += kBlock) {
    const int r = e / I, c = e % I;
    cpx<double> x;
    if (r == c) {
      x = mk(tot[r], 0.0);
    } else {
      const int lo_ = r < c ? r : c, hi_ = r < c ? c : r;
      const int qq = I + 2 * (lo_ * (2 * I - lo_ - 1) / 2 + (hi_ - lo_ - 1));
      x = r < c ? mk(tot[qq], tot[qq + 1]) : mk(tot[qq], -tot[qq + 1]);
    }
    R[2 * e] = x.re / ws;
    R[2 * e + 1] = x.im / ws;
  }
}

// ------------------------------------------------------------ joint diagonaliser
// Dense FP64 complex algebra of one problem in one thread (small local arrays).

// A = L L^H for Hermitian positive definite A (L lower triangular); false if
// a pivot is not positive and finite.
template <int I>
__device__ bool mask_cholesky(const cpx<double> (&A)[I][I], cpx<double> (&L)[I][I]) {
  for (int k = 0; k < I; ++k) {
    double d = A[k][k].re;
    for (int t = 0; t < k; ++t) d -= cabs2(L[k][t]);
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double lk = sqrt(d);
    L[k][k] = mk(lk, 0.0);
    for (int r = k + 1; r < I; ++r) {
      cpx<double> s = A[r][k];
      for (int t = 0; t < k; ++t) s = csub(s, cmul(L[r][t], cconj(L[k][t])));
      L[r][k] = cscale(s, 1.0 / lk);
    }
    for (int c = k + 1; c < I; ++c) L[k][c] = mk(0.0, 0.0);
  }
  return true;
}

// x <- A^{-1} b by Gaussian elimination with partial pivoting (A is
// overwritten); false if a pivot vanishes.
template <int I>
__device__ bool mask_solve(cpx<double> (&A)[I][I], cpx<double> (&b)[I]) {
  for (int k = 0; k < I; ++k) {
    int p = k;
    double best = cabs2(A[k][k]);
    for (int r = k + 1; r < I; ++r)
      if (cabs2(A[r][k]) > best) {
        best = cabs2(A[r][k]);
        p = r;
      }
    if (!(best > 0.0) || !isfinite(best)) return false;
    if (p != k) {
      for (int c = 0; c < I; ++c) {
        const cpx<double> t = A[k][c];
        A[k][c] = A[p][c];
        A[p][c] = t;
      }
      const cpx<double> t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
    const cpx<double> inv = cscale(cconj(A[k][k]), 1.0 / best);
    for (int r = k + 1; r < I; ++r) {
      const cpx<double> l = cmul(A[r][k], inv);
      for (int c = k; c < I; ++c) A[r][c] = csub(A[r][c], cmul(l, A[k][c]));
      b[r] = csub(b[r], cmul(l, b[k]));
    }
  }
  for (int k = I - 1; k >= 0; --k) {
    cpx<double> s = b[k];
    for (int c = k + 1; c < I; ++c) s = csub(s, cmul(A[k][c], b[c]));
    b[k] = cmul(s, cscale(cconj(A[k][k]), 1.0 / cabs2(A[k][k])));
  }
  return true;
}

// Eigen-decomposition W = U diag(w) U^H of a Hermitian W by cyclic Jacobi
// rotations (W is overwritten by diag(w)): for each pair p < q with
// W_pq = r e^{i phi}, the unitary Z = diag(1, e^{-i phi}) G, G the real
// rotation with t = tan(theta) = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (W_qq - W_pp) / (2 r), sets W_pq to zero (W <- Z^H W Z, U <- U Z).
template <int I>
__device__ void mask_jacobi(cpx<double> (&W)[I][I], cpx<double> (&U)[I][I]) {
  for (int r = 0; r < I; ++r)
    for (int c = 0; c < I; ++c) U[r][c] = mk(r == c ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int r = 0; r < I; ++r)
      for (int c = 0; c < I; ++c) {
        all += cabs2(W[r][c]);
        if (r != c) off += cabs2(W[r][c]);
      }
    if (!(off > 1e-32 * all)) break;
    for (int p = 0; p < I; ++p)
      for (int q = p + 1; q < I; ++q) {
        const double r2 = cabs2(W[p][q]);
        if (!(r2 > 0.0)) continue;
        const double rr = sqrt(r2);
        const cpx<double> e = cscale(cconj(W[p][q]), 1.0 / rr);  // e^{-i phi}
        const double tau = (W[q][q].re - W[p][p].re) / (2.0 * rr);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        const cpx<double> se = cscale(e, s), ce = cscale(e, c);  // s e^{-i phi}, c e^{-i phi}
        for (int k = 0; k < I; ++k) {  // columns p, q of W and U: (x, y) Z
          const cpx<double> x = W[k][p], y = W[k][q];
          W[k][p] = csub(cscale(x, c), cmul(se, y));
          W[k][q] = cadd(cscale(x, s), cmul(ce, y));
          const cpx<double> u = U[k][p], v = U[k][q];
          U[k][p] = csub(cscale(u, c), cmul(se, v));
          U[k][q] = cadd(cscale(u, s), cmul(ce, v));
        }
        for (int k = 0; k < I; ++k) {  // rows p, q of W: Z^H (x, y)
          const cpx<double> x = W[p][k], y = W[q][k];
          W[p][k] = csub(cscale(x, c), cmul(cconj(se), y));
          W[q][k] = cadd(cscale(x, s), cmul(cconj(ce), y));
        }
        W[p][q] = W[q][p] = mk(0.0, 0.0);
        W[p][p].im = W[q][q].im = 0.0;
      }
  }
}

// lambda_ji = p_i^H R_j p_i for every j, i (R_j from the workspace).
template <int I>
__device__ void mask_powers(const double* R, int J, const cpx<double> (&P)[I][I], double (&lam)[kMaskMaxJ][I]) {
  for (int j = 0; j < J; ++j) {
    const cpx<double>* Rj = reinterpret_cast<const cpx<double>*>(R) + (size_t)j * I * I;
    for (int i = 0; i < I; ++i) {
      double s = 0.0;
      for (int a = 0; a < I; ++a) {
        cpx<double> t = mk(0.0, 0.0);
        for (int b = 0; b < I; ++b) t = cadd(t, cmul(Rj[a * I + b], P[b][i]));
        s += P[a][i].re * t.re + P[a][i].im * t.im;  // Re(conj(P_ai) t)
      }
      lam[j][i] = s;
    }
  }
}

template <int I>
__global__ void __launch_bounds__(64) k_mask_ajd(MaskArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.part.F) return;
  const int J = a.J;
  const double* R = a.R + (size_t)p * J * I * I * 2;
  const cpx<double>* Rc = reinterpret_cast<const cpx<double>*>(R);
  bool bad = false;
  // the start: generalized eigenvectors of (R_1, R_y)
  cpx<double> A[I][I], L[I][I], W[I][I], U[I][I], P[I][I];
  for (int r = 0; r < I; ++r)
    for (int c = 0; c < I; ++c) {
      cpx<double> s = mk(0.0, 0.0);
      for (int j = 0; j < J; ++j) s = cadd(s, Rc[((size_t)j * I + r) * I + c]);
      A[r][c] = s;
    }
  bad |= !mask_cholesky<I>(A, L);
  for (int c = 0; c < I; ++c)  // A <- L^{-1} (forward substitution, column by column)
    for (int r = 0; r < I; ++r) {
      cpx<double> s = mk(r == c ? 1.0 : 0.0, 0.0);
      for (int t = c; t < r; ++t) s = csub(s, cmul(L[r][t], A[t][c]));
      A[r][c] = r < c ? mk(0.0, 0.0) : cscale(s, 1.0 / L[r][r].re);
    }
  for (int r = 0; r < I; ++r)  // W = L^{-1} R_1 L^{-H}
    for (int c = 0; c < I; ++c) {
      cpx<double> s = mk(0.0, 0.0);
      for (int x = 0; x < I; ++x) {
        cpx<double> t = mk(0.0, 0.0);
        for (int y = 0; y < I; ++y) t = cadd(t, cmul(Rc[x * I + y], cconj(A[c][y])));
        s = cadd(s, cmul(A[r][x], t));
      }
      W[r][c] = s;
    }
  mask_jacobi<I>(W, U);
  for (int k = 0; k < I; ++k) {  // ascending eigenvalues (selection sort of the columns)
    int best = k;
    for (int c = k + 1; c < I; ++c)
      if (W[c][c].re < W[best][best].re) best = c;
    if (best != k) {
      const cpx<double> t = W[k][k];
      W[k][k] = W[best][best];
      W[best][best] = t;
      for (int r = 0; r < I; ++r) {
        const cpx<double> u = U[r][k];
        U[r][k] = U[r][best];
        U[r][best] = u;
      }
    }
  }
  for (int r = 0; r < I; ++r)  // P = L^{-H} U
    for (int c = 0; c < I; ++c) {
      cpx<double> s = mk(0.0, 0.0);
      for (int b = 0; b < I; ++b) s = cadd(s, cmul(cconj(A[b][r]), U[b][c]));
      P[r][c] = s;
    }
  for (int c = 0; c < I; ++c) {  // each column's entry of largest magnitude real and positive
    int k = 0;
    for (int r = 1; r < I; ++r)
      if (cabs2(P[r][c]) > cabs2(P[k][c])) k = r;
    const double m2 = cabs2(P[k][c]);
    const cpx<double> ph = cscale(cconj(P[k][c]), 1.0 / sqrt(m2));
    for (int r = 0; r < I; ++r) P[r][c] = cmul(P[r][c], ph);
  }
  // alternations: Lambda from P, then Eq. FPI with V_i = (1/J) sum_j R_j / lambda_ji
  double lam[kMaskMaxJ][I];
  for (int sweep = 0; sweep < a.sweeps; ++sweep) {
    mask_powers<I>(R, J, P, lam);
    cpx<double> Q[I][I];  // P^{-H}, column by column
    for (int c = 0; c < I; ++c) {
      cpx<double> x[I];
      for (int r = 0; r < I; ++r) {
        x[r] = mk(r == c ? 1.0 : 0.0, 0.0);
        for (int k = 0; k < I; ++k) A[r][k] = cconj(P[k][r]);  // P^H
      }
      bad |= !mask_solve<I>(A, x);  // P^H x = e_c: x is column c of P^{-H}
      for (int r = 0; r < I; ++r) Q[r][c] = x[r];
    }
    for (int i = 0; i < I; ++i) {
      cpx<double> x[I];
      for (int r = 0; r < I; ++r) {
        x[r] = Q[r][i];
        for (int c = 0; c < I; ++c) {
          cpx<double> s = mk(0.0, 0.0);
          for (int j = 0; j < J; ++j) s = cadd(s, cscale(Rc[((size_t)j * I + r) * I + c], 1.0 / (J * lam[j][i])));
          A[r][c] = s;
        }
      }
      bad |= !mask_solve<I>(A, x);
      for (int r = 0; r < I; ++r) W[r][i] = x[r];  // the new column i (W as scratch)
    }
    for (int r = 0; r < I; ++r)
      for (int c = 0; c < I; ++c) P[r][c] = W[r][c];
  }
  mask_powers<I>(R, J, P, lam);
  for (int j = 0; j < J; ++j)
    for (int i = 0; i < I; ++i) {
      bad |= !(lam[j][i] > 0.0) || !isfinite(lam[j][i]);
      a.lam[((size_t)p * J + j) * I + i] = lam[j][i];
    }
  for (int r = 0; r < I; ++r)
    for (int c = 0; c < I; ++c) {
      a.P[(((size_t)p * I + r) * I + c) * 2] = P[r][c].re;
      a.P[(((size_t)p * I + r) * I + c) * 2 + 1] = P[r][c].im;
    }
  if (bad) raise_status(a.status, kDevSingular, p);
}

// ------------------------------------------------------------ source powers
template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_mask_v(MaskArgs a) {
  using C = cpx<T>;
  __shared__ cpx<T> sP[I][I];
  __shared__ T sRl[kMaskMaxJ][I];  // 1 / (I lambda_ji)
  const int p = blockIdx.x;
  const Partition& pt = a.part;
  const int n = pt.frames(p);
  const long long rlen = pt.row_len(p, a.ld), off = pt.frame_off(p), fr = pt.freq(p);
  const size_t rs = (size_t)pt.Fm * rlen;
  const C* y = reinterpret_cast<const C*>(a.y) + (size_t)a.I * pt.Fm * off + fr * rlen;
  const T* m = reinterpret_cast<const T*>(a.m) + (size_t)a.J * pt.Fm * off + fr * rlen;
  T* v = reinterpret_cast<T*>(a.v) + (size_t)a.J * pt.Fm * off + fr * rlen;
  for (int e = threadIdx.x; e < I * I; e += kBlock)
    sP[e / I][e % I] = mk<T>((T)a.P[((size_t)p * I * I + e) * 2], (T)a.P[((size_t)p * I * I + e) * 2 + 1]);
  for (int e = threadIdx.x; e < a.J * I; e += kBlock)
    sRl[e / I][e % I] = (T)(1.0 / ((double)I * a.lam[(size_t)p * a.J * I + e]));
  __syncthreads();
  const T delta = (T)a.delta;
  for (int t = threadIdx.x; t < n; t += kBlock) {
    T e2[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
      C s = mk<T>(0, 0);
#pragma unroll
      for (int r = 0; r < I; ++r) cfmac(s, sP[r][i], y[r * rs + t]);  // conj(P_ri) y_r
      e2[i] = cabs2(s);
    }
    for (int j = 0; j < a.J; ++j) {
      T q = 0;
#pragma unroll
      for (int i = 0; i < I; ++i) q = fma(e2[i], sRl[j][i], q);
      const T mj = m[j * rs + t];
      v[j * rs + t] = (mj > delta ? mj : delta) * q;
    }
  }
}

}  // namespace ffca
