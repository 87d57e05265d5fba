// Per-problem FP64 kernels of the P step by elimination (used from four
// microphones up, where the cofactor forms of k_psolve take more FP64
// instructions), and the Wiener filter for more than four microphones.
// Lane (g, c) of a warp owns column c of problem g (32 / I problems per
// warp) and every matrix lives in registers, distributed by columns over
// the problem's I lanes:
//
//   k_psolve_ldl  Eq. FPI: each lane factors its V_i = L D L^H (right-looking,
//                 no square roots) and solves V_i p_i = [P^{-H}]_i with the
//                 P^{-H} of the current P (kept in the workspace from the
//                 step that made P); K sweeps, all columns from one P^{-H}
//                 per sweep; then the in-place Gauss-Jordan inverse of the
//                 new P^H gives ln|det P|^2 for the next log-likelihood and
//                 the next P^{-H}.
//   k_prep_gj     ln|det P|^2, P^{-H} and the pass-A table of the current P.
//   k_wiener_big  Eq. MMSE0 for I > 4.
//
// On this part an FP64 warp instruction occupies the SM's FP64 pipe for 16
// cycles (2 FP64 FMAs per clock per SM), so the kernels count FP64
// instructions: pivot choices use integer compares of the magnitudes' bit
// patterns, the in-place inverse updates one I x I matrix per step (not an
// augmented I x 2I one), and the inverse of P is carried from one step to
// the next instead of being recomputed.
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

template <int I>
struct BigLane {
  static constexpr int G = 32 / I;  // problems per warp
  static constexpr int LDM = I + 1; // padded row of the transpose buffer (conflict-free column reads)
  // per block (one warp): each problem's I x I matrix for transposes, plus
  // one for the idle lanes (32 % I of them)
  static constexpr int SMEM = (G + 1) * I * LDM * (int)sizeof(cpx<double>);
};

// Pivot key: max(|re|, |im|) compared through the bit patterns of the
// absolute values (monotonic for non-negative doubles), within a factor
// sqrt(2) of |z|: enough to choose a partial pivot, with integer compares
// instead of FP64 instructions.
__device__ inline unsigned long long pivot_key(cpx<double> z) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(z.re) & 0x7fffffffffffffffull;
  const unsigned long long b = (unsigned long long)__double_as_longlong(z.im) & 0x7fffffffffffffffull;
  return a > b ? a : b;
}

// In-place Gauss-Jordan inverse with partial pivoting of the I x I complex
// matrix whose column c lane (g, c) holds in a[] (rows 0..I-1); on return
// a[] holds column c of the inverse.  Step k: the owner of column k picks
// the pivot row p >= k, every lane swaps rows k and p of its column, the
// pivot column is broadcast, and with t = a_k / pivot (t = 1 / pivot for the
// owner) each lane sets a_k = t and a_r -= col_r t (r != k; the owner starts
// from 0).  The row interchanges of steps k become column interchanges of
// the result, undone in reverse order by one gather at the end.  Returns
// |det|^2 as the product of the pivots' |.|^2 (0 if a pivot vanished).
template <int I>
__device__ double gj_inverse_cols(cpx<double> (&a)[I], int g, int c) {
  const unsigned full = 0xffffffffu;
  int perm[I];
  double det2 = 1.0;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const int owner = g * I + k;
    int p = k;
    unsigned long long best = pivot_key(a[k]);
#pragma unroll
    for (int r = k + 1; r < I; ++r) {
      const unsigned long long m = pivot_key(a[r]);
      if (m > best) {
        best = m;
        p = r;
      }
    }
    p = __shfl_sync(full, p, owner);
    perm[k] = p;
#pragma unroll
    for (int r = k + 1; r < I; ++r) {
      if (r == p) {
        const cpx<double> t = a[k];
        a[k] = a[r];
        a[r] = t;
      }
    }
    cpx<double> col[I];
#pragma unroll
    for (int r = 0; r < I; ++r) col[r] = shfl_c(a[r], owner);
    const double d2 = cabs2(col[k]);
    det2 *= d2;
    const double rd = recip(d2);
    const cpx<double> inv = mk(col[k].re * rd, -col[k].im * rd);
    const bool piv = (c == k);
    const cpx<double> t = piv ? inv : cmul(a[k], inv);
#pragma unroll
    for (int r = 0; r < I; ++r) {
      if (r == k) continue;
      cpx<double> v = piv ? mk(0.0, 0.0) : a[r];
      cfma(v, mk(-col[r].re, -col[r].im), t);
      a[r] = v;
    }
    a[k] = t;
  }
  // column c of the result is column sigma(c) of the matrix before the
  // interchanges: trace the swaps (k, perm[k]), applied for k = I-1 .. 0
  int j = c;
#pragma unroll
  for (int k = 0; k < I; ++k) j = (j == k) ? perm[k] : (j == perm[k] ? k : j);
#pragma unroll
  for (int r = 0; r < I; ++r) a[r] = shfl_c(a[r], g * I + j);
  return (det2 > 0.0 && isfinite(det2)) ? det2 : 0.0;
}

// Index of the strictly lower entry (r, c), r > c, in packed row order.
__host__ __device__ constexpr int lo_index(int r, int c) { return r * (r - 1) / 2 + c; }

// V = L D L^H in place (right-looking, no square roots): on entry dv holds
// the real diagonal and lo the strictly lower entries of the Hermitian V; on
// return lo holds the unit lower factor L and rd the reciprocals of D.
// Returns false if a pivot is at or below kCholRtol times its original
// diagonal entry, or not finite (rank deficient or non-finite V).
template <int I>
__device__ bool ldl_factor(double (&dv)[I], cpx<double> (&lo)[I * (I - 1) / 2], double (&rd)[I]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const double d = dv[k];
    ok &= isfinite(d) && d > 0.0;
    const double inv = recip(d);
    rd[k] = inv;
    cpx<double> l[I];
#pragma unroll
    for (int r = k + 1; r < I; ++r) l[r] = cscale(lo[lo_index(r, k)], inv);
#pragma unroll
    for (int c = k + 1; c < I; ++c) {
      const cpx<double> vck = lo[lo_index(c, k)];
      dv[c] -= vck.re * l[c].re + vck.im * l[c].im;  // |V_ck|^2 / d
#pragma unroll
      for (int r = c + 1; r < I; ++r) {  // V_rc -= V_rk conj(l_c)
        cpx<double>& v = lo[lo_index(r, c)];
        const cpx<double> vrk = lo[lo_index(r, k)];
        v = csub(v, cmul(vrk, cconj(l[c])));
      }
    }
#pragma unroll
    for (int r = k + 1; r < I; ++r) lo[lo_index(r, k)] = l[r];
  }
  return ok;
}

// x <- (L D L^H)^{-1} x with the factors of ldl_factor.
template <int I>
__device__ void ldl_solve(const cpx<double> (&lo)[I * (I - 1) / 2], const double (&rd)[I], cpx<double> (&x)[I]) {
#pragma unroll
  for (int k = 0; k < I; ++k)  // L z = x
#pragma unroll
    for (int r = k + 1; r < I; ++r) cfma(x[r], mk(-lo[lo_index(r, k)].re, -lo[lo_index(r, k)].im), x[k]);
#pragma unroll
  for (int k = 0; k < I; ++k) x[k] = cscale(x[k], rd[k]);
#pragma unroll
  for (int k = I - 1; k >= 0; --k)  // L^H p = z
#pragma unroll
    for (int r = 0; r < k; ++r) {
      const cpx<double> l = lo[lo_index(k, r)];  // (L^H)_rk = conj(L_kr)
      cfma(x[r], mk(-l.re, l.im), x[k]);
    }
}

// Complex arithmetic that the compiler may not contract or fuse: every
// product and sum rounded as written.  The cofactor inverse below is formed
// by kernels that lay out its terms differently (one lane per column, or
// one lane per entry) and must agree bit for bit.
__device__ inline cpx<double> cmul_rn(cpx<double> a, cpx<double> b) {
  return mk(__fma_rn(a.re, b.re, -__dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re)));
}
__device__ inline cpx<double> cadd_rn(cpx<double> a, cpx<double> b) {
  return mk(__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im));
}
__device__ inline cpx<double> csub_rn(cpx<double> a, cpx<double> b) {
  return mk(__dsub_rn(a.re, b.re), __dsub_rn(a.im, b.im));
}
__device__ inline double cabs2_rn(cpx<double> a) { return __fma_rn(a.re, a.re, __dmul_rn(a.im, a.im)); }

// The 2 x 2 minor a d - b c of a 3 x 3 cofactor, and the cofactor inverse's
// final values from the cofactor C and det P (rounded as written).
__device__ inline cpx<double> minor2_rn(cpx<double> a, cpx<double> b, cpx<double> c, cpx<double> d) {
  return csub_rn(cmul_rn(a, d), cmul_rn(b, c));
}
__device__ inline cpx<double> inv_from_cofactor(cpx<double> C, cpx<double> det, double rd2) {
  const cpx<double> rdet = mk(__dmul_rn(det.re, rd2), -__dmul_rn(det.im, rd2));  // 1 / det
  return cconj(cmul_rn(C, rdet));
}

// Column c of P^{-H} and |det P|^2 from the columns of P (lane (g, c) holds
// column c of P in x[]), for I <= 4 by cofactors: one division instead of I
// dependent pivot steps.  The lane gathers P with its columns rotated,
// A[:, k] = P[:, (c + k) mod I], so that column c of the cofactor matrix is
// column 0 of A's, up to the sign (-1)^(c (I-1-c)) of the rotation of the
// other columns; then (P^{-H})_{rc} = conj(C_rc / det P) with det P the
// expansion along column 0 of lane (g, 0), shared by the problem's lanes.
template <int I>
__device__ double pinvh_cofactors(cpx<double> (&x)[I], int g, int c, bool& singular) {
  static_assert(I <= 4, "cofactor forms for I <= 4");
  cpx<double> A[I][I];
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const int src = g * I + (c + k) % I;
#pragma unroll
    for (int r = 0; r < I; ++r) A[r][k] = shfl_c(x[r], src);
  }
  const bool flip = ((c * (I - 1 - c)) & 1) != 0;
  cpx<double> C[I];
  cpx<double> det = mk(0.0, 0.0);
#pragma unroll
  for (int r = 0; r < I; ++r) {
    cpx<double> m;
    if constexpr (I == 3) {
      const int r0 = r == 0 ? 1 : 0, r1 = r == 2 ? 1 : 2;  // rows of the minor, columns 1 and 2
      m = minor2_rn(A[r0][1], A[r0][2], A[r1][1], A[r1][2]);
    } else {
      m = minor_det<I>(A, r, 0);
    }
    C[r] = ((((r + c) & 1) != 0) != flip) ? mk(-m.re, -m.im) : m;
    det = cadd_rn(det, cmul_rn(A[r][0], C[r]));
  }
  det = shfl_c(det, g * I);  // the expansion of lane (g, 0), for every lane of the problem
  const double d2 = cabs2_rn(det);
  singular |= !(d2 > 0.0) || !isfinite(d2);
  const double inv = recip(d2);
#pragma unroll
  for (int r = 0; r < I; ++r) x[r] = inv_from_cofactor(C[r], det, inv);
  return (d2 > 0.0 && isfinite(d2)) ? d2 : 0.0;
}

// Column c of P^{-H} and |det P|^2 from the columns of P (lane (g, c) holds
// column c of P in x[]): for I <= 3 by cofactors (the shortest FP64
// dependency chain: 18.7 against 20.4 us per long-mixture P step); else
// transpose through the problem's shared buffer M (rows padded to LDM),
// conjugate into column c of P^H, invert by Gauss-Jordan (fewer FP64
// instructions from I = 4: the batched P step, bound by FP64 throughput,
// takes 181 us against 219 us with the cofactors).
template <int I>
__device__ double pinvh_from_columns(cpx<double> (&x)[I], cpx<double>* M, int g, int c, bool& singular) {
  if constexpr (I <= 3) return pinvh_cofactors<I>(x, g, c, singular);
  constexpr int LDM = BigLane<I>::LDM;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < I; ++r) M[r * LDM + c] = x[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < I; ++r) x[r] = cconj(M[c * LDM + r]);  // (P^H)_{rc} = conj(P_cr)
  const double det2 = gj_inverse_cols<I>(x, g, c);
  singular |= !(det2 > 0.0);
  return det2;
}

// The gradient updates of P (Sec. 4.6) for lane (g, i): on entry dv and lo
// hold V_i (real diagonal, strictly lower entries V_rc, r > c) and x column
// i of P^{-H} of the current P; on return x holds column i of the new P.
// K steps with V_i fixed; the natural gradient forms P (P^H w) one column of
// P at a time, broadcast from its lane.
template <int I>
__device__ void gradient_steps(const FastArgs& a, int f, const double (&dv)[I],
                               const cpx<double> (&lo)[I * (I - 1) / 2], cpx<double> (&x)[I],
                               cpx<double>* M, int g, int i, bool& singular) {
  cpx<double> p[I];  // column i of the current P
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const double2 q = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I * I + r * I + i);
    p[r] = mk(q.x, q.y);
  }
  for (int step = 0; step < a.K; ++step) {
    cpx<double> w[I];  // V_i p_i
#pragma unroll
    for (int r = 0; r < I; ++r) {
      cpx<double> s = mk(dv[r] * p[r].re, dv[r] * p[r].im);
#pragma unroll
      for (int c = 0; c < I; ++c) {
        if (c < r) cfma(s, lo[lo_index(r, c)], p[c]);
        if (c > r) cfmac(s, lo[lo_index(c, r)], p[c]);  // V_rc = conj(V_cr)
      }
      w[r] = s;
    }
    if (a.pmode == kPGradient) {
      if (step > 0) {  // P^{-H} of the intermediate P
#pragma unroll
        for (int r = 0; r < I; ++r) x[r] = p[r];
        pinvh_from_columns<I>(x, M, g, i, singular);
      }
#pragma unroll
      for (int r = 0; r < I; ++r)
        p[r] = mk(p[r].re + a.mu * (x[r].re - w[r].re), p[r].im + a.mu * (x[r].im - w[r].im));
    } else {
      cpx<double> u[I];  // P (P^H w)
#pragma unroll
      for (int r = 0; r < I; ++r) u[r] = mk(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < I; ++k) {
        cpx<double> pk[I];
#pragma unroll
        for (int r = 0; r < I; ++r) pk[r] = shfl_c(p[r], g * I + k);
        cpx<double> ck = mk(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < I; ++r) cfmac(ck, pk[r], w[r]);  // p_k^H w
#pragma unroll
        for (int r = 0; r < I; ++r) cfma(u[r], pk[r], ck);
      }
#pragma unroll
      for (int r = 0; r < I; ++r)
        p[r] = mk(p[r].re + a.mu * (p[r].re - u[r].re), p[r].im + a.mu * (p[r].im - u[r].im));
    }
  }
#pragma unroll
  for (int r = 0; r < I; ++r) x[r] = p[r];
}

// GRAD selects the gradient updates (a separate kernel, so that the
// fixed-point one keeps its registers).
template <typename T, int I, int J, bool GRAD = false>
__global__ void __launch_bounds__(32) k_psolve_ldl(FastArgs a) {
  using BL = BigLane<I>;
  constexpr int G = BL::G;
  constexpr int NV = I * I * I;
  constexpr int NL = I * (I - 1) / 2;
  extern __shared__ __align__(16) unsigned char big_smem[];
  if (trace_block(a)) return;
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f0 = blockIdx.x * G + g;
  const bool active = g < G && f0 < a.F;
  const int f = active ? f0 : 0;  // idle lanes shadow problem 0 and write nothing
  cpx<double>* M = reinterpret_cast<cpx<double>*>(big_smem) + (size_t)(g < G ? g : G) * I * BL::LDM;
  const Partition pt = a.part;

  // every global load first, all independent of one another: the new
  // Lambda, column i of P^{-H} of the current P, and the slots of V_i
  // (packed Hermitian: diagonal, then (re, im) above it in row order; 16-byte
  // loads where the I^2 values of each i start on a 16-byte boundary)
  double lnext[J];
  if (a.lam_next) {
#pragma unroll
    for (int j = 0; j < J; ++j) lnext[j] = __ldcg(a.lam_next + (size_t)f * J * I + j * I + i);
  }
  cpx<double> x[I];
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const double2 q = __ldcg(reinterpret_cast<const double2*>(a.pinvH) + (size_t)f * I * I + r * I + i);
    x[r] = mk(q.x, q.y);
  }
  double dv[I], rd[I];
  cpx<double> lo[NL];
  {
    double pk[I * I];
    const int ns = pt.nslots(f);  // >= 1: every problem has a slot
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV + i * I * I;
    if constexpr ((I * I) % 2 == 0) {
      const double2* b2 = reinterpret_cast<const double2*>(base);
#pragma unroll
      for (int m = 0; m < I * I / 2; ++m) {
        const double2 v2 = __ldcg(b2 + m);
        pk[2 * m] = v2.x;
        pk[2 * m + 1] = v2.y;
      }
      for (int k = 1; k < ns; ++k) {
#pragma unroll
        for (int m = 0; m < I * I / 2; ++m) {
          const double2 v2 = __ldcg(b2 + (size_t)k * (NV / 2) + m);
          pk[2 * m] += v2.x;
          pk[2 * m + 1] += v2.y;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < I * I; ++m) pk[m] = __ldcg(base + m);
      for (int k = 1; k < ns; ++k)
#pragma unroll
        for (int m = 0; m < I * I; ++m) pk[m] += __ldcg(base + (size_t)k * NV + m);
    }
    if (active && a.lam_next) {  // commit the new Lambda (computed during pass B)
      ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        a.lam[(size_t)f * J * I + j * I + i] = lnext[j];
        ta->set_lam(j, i, (T)lnext[j]);
      }
    }
    const double sc = pt.inv_n(f);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < I * I; ++m) {
      pk[m] *= sc;
      bad |= !isfinite(pk[m]);
    }
    if (active && bad) raise_status(a.status, kDevNonfinite, f);
#pragma unroll
    for (int r = 0; r < I; ++r) dv[r] = pk[r];
    int m = I;
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = r + 1; c < I; ++c) {
        lo[lo_index(c, r)] = mk(pk[m], -pk[m + 1]);  // V_cr = conj(V_rc)
        m += 2;
      }
  }
  bool singular = false;
  if constexpr (GRAD) {
    gradient_steps<I>(a, f, dv, lo, x, M, g, i, singular);
  } else {
    double d0[I];
#pragma unroll
    for (int r = 0; r < I; ++r) d0[r] = dv[r];
    singular = !ldl_factor<I>(dv, lo, rd);
#pragma unroll
    for (int r = 0; r < I; ++r) singular |= !(dv[r] > kCholRtol * d0[r]);  // dv holds the pivots D
    for (int sweep = 0; sweep < a.K; ++sweep) {
      ldl_solve<I>(lo, rd, x);  // p_i = V_i^{-1} [P^{-H}]_i
      if (sweep + 1 < a.K) pinvh_from_columns<I>(x, M, g, i, singular);  // P^{-H} of the intermediate P
    }
  }
  double det2 = 0.0;
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int r = 0; r < I; ++r) {
      reinterpret_cast<double2*>(a.P)[(size_t)f * I * I + r * I + i] = make_double2(x[r].re, x[r].im);
      ta->set_p(r, i, (T)x[r].re, (T)x[r].im);
    }
  }
  // the next step's P^{-H} and ln|det P|^2 of the new P (Eq. L2)
  det2 = pinvh_from_columns<I>(x, M, g, i, singular);
  if (active) {
#pragma unroll
    for (int r = 0; r < I; ++r)
      reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I * I + r * I + i] = make_double2(x[r].re, x[r].im);
    if (singular) raise_status(a.status, kDevSingular, f);
    if (i == 0) {
      atomicAdd(a.ops, p_update_inversions(a, I));
      a.logdet[f] = log(det2);
    }
  }
}

// ln|det P|^2, P^{-H} (always: the P step starts from it) and the pass-A
// table of the current P and Lambda.  P^{-H} is formed by the same routine
// (pinvh_from_columns) as the P step's carried one, so iterating in one call
// or in several gives the same bits.
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_prep_gj(FastArgs a) {
  using BL = BigLane<I>;
  constexpr int G = BL::G;
  extern __shared__ __align__(16) unsigned char big_smem[];
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f0 = blockIdx.x * G + g;
  const bool active = g < G && f0 < a.F;
  const int f = active ? f0 : 0;
  cpx<double>* M = reinterpret_cast<cpx<double>*>(big_smem) + (size_t)(g < G ? g : G) * I * BL::LDM;
  cpx<double> x[I];  // column i of P
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const double2 q = reinterpret_cast<const double2*>(a.P)[(size_t)f * I * I + r * I + i];
    x[r] = mk(q.x, q.y);
  }
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int r = 0; r < I; ++r) ta->set_p(r, i, (T)x[r].re, (T)x[r].im);
#pragma unroll
    for (int j = 0; j < J; ++j) ta->set_lam(j, i, (T)a.lam[(size_t)f * J * I + j * I + i]);
  }
  bool singular = false;
  const double det2 = pinvh_from_columns<I>(x, M, g, i, singular);
  if (!active) return;
  if (singular) raise_status(a.status, kDevSingular, f);
  if (i == 0) a.logdet[f] = log(det2);
  if (a.pinvH) {
#pragma unroll
    for (int r = 0; r < I; ++r)
      reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I * I + r * I + i] = make_double2(x[r].re, x[r].im);
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
  const long long u0 = pt.block_start(blockIdx.x);
  const long long u1 = pt.block_start(blockIdx.x + 1);
  const long long row = a.ld / FU;

  for (long long u = u0; u < u1;) {
    const int f = pt.problem_of(u);
    const long long us = pt.start(f);
    const int k0 = (int)(u - us);
    const int k1 = (int)(min(pt.start(f + 1), u1) - us);
    const int Np = pt.frames(f);
    const long long rlen = pt.row_len(f, row * FU) / FU;
    const long long off = pt.frame_off(f) / FU;
    const long long r0 = (long long)pt.freq(f) * rlen;
    const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y) + (size_t)I * pt.Fm * off + r0;
    const VV* __restrict__ v = reinterpret_cast<const VV*>(a.v) + (size_t)J * pt.Fm * off + r0;
    VY* __restrict__ out = reinterpret_cast<VY*>(a.out) + (size_t)J * I * pt.Fm * off + r0;
    const size_t rstr = (size_t)pt.Fm * rlen;
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
      for (int j = 0; j < J; ++j) vu[j] = v[j * rstr + k];
      {
        VY yu[I];
#pragma unroll
        for (int m = 0; m < I; ++m) yu[m] = y[m * rstr + k];
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
          const bool valid = k * FU + e < Np;
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
        for (int r = 0; r < I; ++r) out[(j * I + r) * rstr + k] = o[r];
      }
    }
    u += k1 - k0;
  }
}

}  // namespace ffca
