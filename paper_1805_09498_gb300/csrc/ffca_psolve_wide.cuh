// The P step of Eq. FPI with one warp per problem, for I = 3, 4 and 8.
//
// An FP64 warp instruction occupies its SM sub-partition's FP64 unit for 64
// cycles on this part (2 FP64 FMAs per clock per SM, 4 sub-partitions), with
// any number of active lanes.  The packed forms (k_psolve_ldl: 32 / I
// problems per warp, lane (g, i) factoring and solving its own V_i) issue
// about 1500 (I = 8) or 250 (I = 3) FP64 instructions per warp on 130 or 52
// warps for 513 problems: one warp per SM at most, three of every four
// sub-partitions idle, the time set by one warp's dependent chain.  Here
// each problem has a warp of its own, lane (i, q) = (lane % I, lane / I) for
// q < Q (Q = 4 at I = 8, else I; the other lanes only join the shuffles),
// and the work inside each matrix is spread over the lanes:
//
//   L D L^H of V_i   the Q lanes of V_i share the entries of each step's
//                    trailing triangle (row-major order, entry q + Q m);
//                    the matrices live in shared memory;
//   the solves       V_i p_i = [P^{-H}]_i, rows of each substitution step
//                    over the Q lanes;
//   P^{-H}           I = 8: Gauss-Jordan with partial pivoting on P^H, lane
//                    (c, h) holding rows h and h + 4 of column c
//                    (gj_inverse_wide8); I = 4: the same, one entry per
//                    lane (gj_inverse_wide4); I = 3: cofactors, one per lane
//                    (pinvh_wide3).  Every entry takes the same operations,
//                    in the same order, as in gj_inverse_cols and
//                    pinvh_cofactors (the routines of k_prep_gj and the
//                    other P updates), so the P^{-H} carried to the next
//                    step has the same bits as the one recomputed from P at
//                    the start of a call.
//
// A warp issues fewer FP64 instructions than a packed warp, on shorter
// chains, and the 513 warps of a 513-problem step use every sub-partition.
// Per problem the FP64 work is larger, so the packed forms stay in use for
// many problems (the host picks by the problem count).  The factorisation,
// substitution and P^{-H} helpers here also serve the EM step with one warp
// per problem (k_psolve_em_wide) and the resident form's P step at I = 3.
#pragma once

#include "ffca_big.cuh"

namespace ffca {

template <int I>
struct WideP {
  static_assert(I == 3 || I == 4 || I == 8, "the wide P step is laid out for I = 3, 4 and 8");
  static constexpr int Q = I == 8 ? 4 : I;   // lanes per matrix (lanes I Q and up idle)
  static constexpr int R = (I + Q - 1) / Q;  // rows of a column per lane (2 at I = 8, else 1)
  static constexpr int VS = I * I + 1;       // stride of one V_i (complex entries; the pad skews the banks)
  static constexpr int XS = I + 1;           // stride of one vector
  static constexpr int NV = I * I * I;       // values per slot of pass B's partial sums
};

// Entry e of a lower triangle (diagonal included) in row-major order:
// (0,0), (1,0), (1,1), (2,0), ...  The first s(s+1)/2 entries are those of
// the s x s triangle, whatever its size.
__device__ inline void tri_decode(int e, int& r, int& c) {
  r = 0;
  while (e > r) {
    e -= r + 1;
    ++r;
  }
  c = e;
}

// Packed order of the upper entries (r < c) of pass B's slots: row order.
// p < I (I - 1) / 2; the loop is bounded whatever p is.
template <int I>
__device__ inline void upper_decode(int p, int& r, int& c) {
  r = 0;
#pragma unroll
  for (int k = 0; k < I - 2; ++k) {
    if (p >= I - 1 - r) {
      p -= I - 1 - r;
      ++r;
    }
  }
  c = r + 1 + p;
}

// In-place Gauss-Jordan inverse of an 8 x 8 complex matrix A held by the
// whole warp: lane (c, h) = (lane % 8, lane / 8) holds a0 = A[h][c] and
// a1 = A[h + 4][c]; on return the same entries of A^{-1}.  Step k: the
// largest pivot key in column k over rows k .. 7 (the smallest row among
// equal keys, as a first-maximum scan finds), rows k and p exchanged, then
// with t = A[k][c] / pivot (1 / pivot in column k) every other row takes
// A[r][c] - A[r][k] t (0 - A[r][k] t in column k) and row k takes t.  The
// row exchanges become column exchanges of the result, undone at the end.
// Returns |det A|^2 as the product of the pivots' |.|^2 (0 if a pivot
// vanished or the product is not finite).
__device__ inline double gj_inverse_wide8(cpx<double>& a0, cpx<double>& a1, int c, int h) {
  constexpr int I = 8;
  const unsigned full = 0xffffffffu;
  int perm[I];
  double det2 = 1.0;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    unsigned long long key = 0ull;
    int row = I;  // no candidate
    if (h >= k) {
      key = pivot_key(a0);
      row = h;
    }
    if (h + 4 >= k) {
      const unsigned long long k1 = pivot_key(a1);
      if (row == I || k1 > key) {
        key = k1;
        row = h + 4;
      }
    }
#pragma unroll
    for (int s = 8; s <= 16; s <<= 1) {
      const unsigned long long ok = __shfl_xor_sync(full, key, s);
      const int orow = __shfl_xor_sync(full, row, s);
      if (ok > key || (ok == key && orow < row)) {
        key = ok;
        row = orow;
      }
    }
    const int p = __shfl_sync(full, row, k);  // column k's result (lane (k, 0))
    perm[k] = p;
    // entries (k, c) and (p, c) of this lane's column, from the lanes holding them
    const cpx<double> vk = shfl_c(k >= 4 ? a1 : a0, c + 8 * (k & 3));
    const cpx<double> vp = shfl_c(p >= 4 ? a1 : a0, c + 8 * (p & 3));
    if (h == (k & 3)) {
      if (k >= 4) a1 = vp;
      else a0 = vp;
    }
    if (h == (p & 3)) {
      if (p >= 4) a1 = vk;
      else a0 = vk;
    }
    // column k after the exchange: this lane's rows, and the pivot
    const cpx<double> col0 = shfl_c(a0, k + 8 * h);
    const cpx<double> col1 = shfl_c(a1, k + 8 * h);
    const cpx<double> piv = shfl_c(vp, k);
    const double d2 = cabs2(piv);
    det2 *= d2;
    const double rd = recip(d2);
    const cpx<double> inv = mk(piv.re * rd, -piv.im * rd);
    const bool pc = (c == k);
    const cpx<double> t = pc ? inv : cmul(vp, inv);  // vp: entry (k, c) after the exchange
    cpx<double> v0 = pc ? mk(0.0, 0.0) : a0;
    cfma(v0, mk(-col0.re, -col0.im), t);
    cpx<double> v1 = pc ? mk(0.0, 0.0) : a1;
    cfma(v1, mk(-col1.re, -col1.im), t);
    a0 = (h == k) ? t : v0;
    a1 = (h + 4 == k) ? t : v1;
  }
  // column c of the result is column sigma(c) of the matrix before the
  // interchanges: the swaps (k, perm[k]) traced as in gj_inverse_cols
  int j = c;
#pragma unroll
  for (int k = 0; k < I; ++k) j = (j == k) ? perm[k] : (j == perm[k] ? k : j);
  a0 = shfl_c(a0, j + 8 * h);
  a1 = shfl_c(a1, j + 8 * h);
  return (det2 > 0.0 && isfinite(det2)) ? det2 : 0.0;
}

// The same Gauss-Jordan inverse for a 4 x 4 matrix, one entry per lane:
// lane (c, h) = (lane % 4, lane / 4) holds a = A[h][c] for lanes 0 .. 15
// (lanes 16 .. 31 hold nothing of A and only join the shuffles).  Every
// entry takes the operations of gj_inverse_cols<4> in the same order.
__device__ inline double gj_inverse_wide4(cpx<double>& a, int c, int h) {
  constexpr int I = 4;
  const unsigned full = 0xffffffffu;
  int perm[I];
  double det2 = 1.0;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    unsigned long long key = 0ull;
    int row = I;  // no candidate
    if (h >= k && h < I) {
      key = pivot_key(a);
      row = h;
    }
#pragma unroll
    for (int s = 4; s <= 8; s <<= 1) {
      const unsigned long long ok = __shfl_xor_sync(full, key, s);
      const int orow = __shfl_xor_sync(full, row, s);
      if (ok > key || (ok == key && orow < row)) {
        key = ok;
        row = orow;
      }
    }
    const int p = __shfl_sync(full, row, k);  // column k's result (lane (k, 0))
    perm[k] = p;
    const cpx<double> vk = shfl_c(a, c + 4 * k);  // entries (k, c) and (p, c)
    const cpx<double> vp = shfl_c(a, c + 4 * p);
    if (h == k) a = vp;
    if (h == p) a = vk;
    const cpx<double> col = shfl_c(a, k + 4 * (h & 3));  // entry (h, k) after the exchange
    const cpx<double> piv = shfl_c(vp, k);
    const double d2 = cabs2(piv);
    det2 *= d2;
    const double rd = recip(d2);
    const cpx<double> inv = mk(piv.re * rd, -piv.im * rd);
    const bool pc = (c == k);
    const cpx<double> t = pc ? inv : cmul(vp, inv);
    cpx<double> v = pc ? mk(0.0, 0.0) : a;
    cfma(v, mk(-col.re, -col.im), t);
    a = (h == k) ? t : v;
  }
  int j = c;
#pragma unroll
  for (int k = 0; k < I; ++k) j = (j == k) ? perm[k] : (j == perm[k] ? k : j);
  a = shfl_c(a, j + 4 * (h & 3));
  return (det2 > 0.0 && isfinite(det2)) ? det2 : 0.0;
}

// Column c of P^{-H} and |det P|^2 for I = 3 by cofactors, lane (c, r) =
// (lane % 3, lane / 3) for lanes 0 .. 8 (the others shadow row 0), P's
// column c in sX[c][0 .. 2].  Every value takes the operations of
// pinvh_cofactors, each rounded as written (cmul_rn and its kin): with the
// columns of P rotated by c (A[x][k] = P[x][(c + k) mod 3]) the lane forms
// the minor of A without row r and column 0 and its signed cofactor C;
// det P is the expansion along column 0
// of lane c = 0's rotation, with the cofactors of lanes (0, 0 .. 2) in row
// order; the lane's value is (P^{-H})[r][c] = conj(C / det P).
__device__ inline double pinvh_wide3(const cpx<double> (*sX)[WideP<3>::XS], int c, int r, cpx<double>& out) {
  constexpr int I = 3;
  const int rr = r < I ? r : 0;
  const int r0 = rr == 0 ? 1 : 0, r1 = rr == 2 ? 1 : 2;  // rows of the minor
  const int c1 = (c + 1) % I, c2 = (c + 2) % I;         // columns 1, 2 of A
  // P[x][y] = sX[y][x]
  const cpx<double> m = minor2_rn(sX[c1][r0], sX[c2][r0], sX[c1][r1], sX[c2][r1]);
  const bool flip = ((c * (I - 1 - c)) & 1) != 0;
  const cpx<double> C = ((((rr + c) & 1) != 0) != flip) ? mk(-m.re, -m.im) : m;
  // det P = sum_x P[x][0] C_x over lane c = 0's cofactors: lane (0, x)
  // forms term x, every lane sums the terms in row order
  const cpx<double> term = cmul_rn(sX[c][rr], C);
  cpx<double> det = mk(0.0, 0.0);
#pragma unroll
  for (int x = 0; x < I; ++x) det = cadd_rn(det, shfl_c(term, I * x));
  const double d2 = cabs2_rn(det);
  out = inv_from_cofactor(C, det, recip(d2));
  return (d2 > 0.0 && isfinite(d2)) ? d2 : 0.0;
}

// P^{-H} of the P whose column i is sX[i][0 .. I-1] and |det P|^2: lane
// (i, q) receives (P^{-H})[q + Q m][i], m < R.  I = 8 and 4: Gauss-Jordan
// on P^H, (P^H)[x][y] = conj(P[y][x]); I = 3: cofactors.
template <int I>
__device__ inline double pinvh_wide(const cpx<double> (*sX)[WideP<I>::XS], int i, int q,
                                    cpx<double> (&out)[WideP<I>::R]) {
  if constexpr (I == 8) {
    out[0] = cconj(sX[q][i]);
    out[1] = cconj(sX[q + 4][i]);
    return gj_inverse_wide8(out[0], out[1], i, q);
  } else if constexpr (I == 4) {
    out[0] = q < I ? cconj(sX[q][i]) : mk(0.0, 0.0);
    return gj_inverse_wide4(out[0], i, q);
  } else {
    return pinvh_wide3(sX, i, q, out[0]);
  }
}

// L D L^H (right-looking, no square roots) of the I matrices sV[i] in
// place by lanes (i, q), q < Q (the other lanes only join the barriers):
// sV[i] holds V_i's real diagonal and strictly lower entries (row-major,
// stride I); on return its strictly lower part holds the unit factor L_i
// and sRd[i] the reciprocals of D_i.  sL is scratch.  Returns false for a
// pivot at or below kCholRtol times its diagonal entry, or not finite.
// The caller has synchronised the warp after writing sV.
template <int I>
__device__ inline bool wide_ldl(cpx<double> (*sV)[WideP<I>::VS], cpx<double> (*sL)[WideP<I>::XS],
                                double (*sRd)[WideP<I>::XS], int i, int q) {
  constexpr int Q = WideP<I>::Q;
  const bool live = q < Q;
  double d0[I];  // the diagonal before the factorisation
#pragma unroll
  for (int k = 0; k < I; ++k) d0[k] = sV[i][k * (I + 1)].re;

  // L D L^H in place (right-looking, no square roots).  Lane q takes the
  // entries q + Q m of each step's trailing triangle; their places relative
  // to the triangle's corner are the same at every step (the row-major
  // order of a triangle starts with that of every smaller one).
  constexpr int ME = (I * (I - 1) / 2 + Q - 1) / Q;  // entries per lane at the first step
  int e_rc[ME], e_r[ME], e_c[ME];                   // rr * I + cc, rr * I, cc
#pragma unroll
  for (int m = 0; m < ME; ++m) {
    int rr, cc;
    tri_decode(live ? q + Q * m : 0, rr, cc);
    e_rc[m] = rr * I + cc;
    e_r[m] = rr * I;
    e_c[m] = cc;
  }
  cpx<double>* V = sV[i];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const double d = V[k * (I + 1)].re;
    ok &= isfinite(d) && d > 0.0 && d > kCholRtol * d0[k];
    const double inv = recip(d);
    const int NR = I - 1 - k;          // rows below the pivot
    const int NT = NR * (NR + 1) / 2;  // entries of the trailing triangle
    cpx<double> lr[(I - 1 + Q - 1) / Q];  // this lane's rows of the scaled column
#pragma unroll
    for (int m = 0; m < (NR + Q - 1) / Q; ++m) {
      const int r = k + 1 + q + Q * m;
      if (live && r < I) {
        lr[m] = cscale(V[r * I + k], inv);
        sL[i][r] = lr[m];
      }
    }
    if (q == 0) sRd[i][k] = inv;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < (NT + Q - 1) / Q; ++m) {
      if (live && q + Q * m < NT) {  // V_rc -= V_rk conj(l_c), k < c <= r (the diagonal's real part is |V_rk|^2 / d)
        const int corner = (k + 1) * (I + 1);  // entry (k + 1, k + 1)
        const cpx<double> vrk = V[corner - 1 + e_r[m]], lc = sL[i][k + 1 + e_c[m]];
        cpx<double> v = V[corner + e_rc[m]];
        v.re = fma(-vrk.re, lc.re, fma(-vrk.im, lc.im, v.re));
        v.im = fma(-vrk.im, lc.re, fma(vrk.re, lc.im, v.im));
        V[corner + e_rc[m]] = v;
      }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < (NR + Q - 1) / Q; ++m) {  // column k becomes L's
      const int r = k + 1 + q + Q * m;
      if (live && r < I) V[r * I + k] = lr[m];
    }
  }
  __syncwarp();
  return ok;
}

// x_i <- (L_i D_i L_i^H)^{-1} x_i for the I vectors sX[i], with the factors
// of wide_ldl: the rows of each substitution step over the lanes (i, q).
template <int I>
__device__ inline void wide_solve(const cpx<double> (*sV)[WideP<I>::VS], const double (*sRd)[WideP<I>::XS],
                                  cpx<double> (*sX)[WideP<I>::XS], int i, int q) {
  constexpr int Q = WideP<I>::Q, R = WideP<I>::R;
  const bool live = q < Q;
  const cpx<double>* L = sV[i];
#pragma unroll
  for (int k = 0; k < I - 1; ++k) {  // L z = x
    const cpx<double> zk = sX[i][k];
    const int NR = I - 1 - k;
#pragma unroll
    for (int m = 0; m < (NR + Q - 1) / Q; ++m) {
      const int r = k + 1 + q + Q * m;
      if (live && r < I) {
        const cpx<double> l = L[r * I + k];
        cpx<double> v = sX[i][r];
        cfma(v, mk(-l.re, -l.im), zk);
        sX[i][r] = v;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {  // z = D^{-1} z
    const int r = q + Q * m;
    if (live && r < I) sX[i][r] = cscale(sX[i][r], sRd[i][r]);
  }
  __syncwarp();
#pragma unroll
  for (int k = I - 1; k > 0; --k) {  // L^H p = z: (L^H)_rk = conj(L_kr)
    const cpx<double> zk = sX[i][k];
#pragma unroll
    for (int m = 0; m < (k + Q - 1) / Q; ++m) {
      const int r = q + Q * m;
      if (live && r < k) {
        const cpx<double> l = L[k * I + r];
        cpx<double> v = sX[i][r];
        cfma(v, mk(-l.re, l.im), zk);
        sX[i][r] = v;
      }
    }
    __syncwarp();
  }
}

// k_psolve_wide: one P step of Eq. FPI (K sweeps) for I = 3 or 8, one warp
// per problem (blocks of 32 threads; with a trace the last block sums it).
// The outputs are those of k_psolve_ldl: the new Lambda committed, P and
// its pass-A table, P^{-H}, ln|det P|^2, the inversion count and the status.
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_psolve_wide(FastArgs a) {
  using W = WideP<I>;
  constexpr int Q = W::Q, R = W::R;
  __shared__ cpx<double> sV[I][W::VS];   // V_i, then its unit lower factor L_i (row-major, lower part)
  __shared__ cpx<double> sX[I][W::XS];   // column i of P^{-H}, then p_i
  __shared__ cpx<double> sL[I][W::XS];   // scaled column k of the factorisation step
  __shared__ double sRd[I][W::XS];       // 1 / D of L_i D_i L_i^H
  if (trace_block(a)) return;
  const int f = blockIdx.x;
  if (f >= a.F) return;
  const int lane = threadIdx.x;
  const int i = lane % I, q = lane / I;  // matrix / column i and its lane q (as (c, h) in the inverse)
  const bool live = q < Q;               // lanes I Q and up only join the shuffles
  const Partition pt = a.part;

  // every global load first: the new Lambda, column i of P^{-H} (rows
  // q + Q m) and the slots of the V_i
  constexpr int JL = (J + Q - 1) / Q;
  double lnext[JL];
  if (a.lam_next) {
#pragma unroll
    for (int m = 0; m < JL; ++m) {
      const int j = q + Q * m;
      lnext[m] = live && j < J ? __ldcg(a.lam_next + (size_t)f * J * I + j * I + i) : 0.0;
    }
  }
  cpx<double> xr[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int r = q + Q * m;
    double2 u = make_double2(0.0, 0.0);
    if (live && r < I) u = __ldcg(reinterpret_cast<const double2*>(a.pinvH) + (size_t)f * I * I + r * I + i);
    xr[m] = mk(u.x, u.y);
  }
  const int ns = pt.nslots(f);  // >= 1: every problem has a slot
  const double* slots = a.part_buf + (size_t)f * pt.max_slots * W::NV;
  bool bad = false;
  if constexpr (I % 2 == 0) {
    // lane (i, q): I I / (2 Q) 16-byte units of V_i's packed values (I
    // diagonal values, then (re, im) of V_rc, r < c, in row order)
    // (lanes q >= Q, present at I = 4, hold no units)
    constexpr int U = I * I / 2 / Q;
    double2 pk[U];
    const double2* b2 = reinterpret_cast<const double2*>(slots + i * I * I) + (live ? q : 0) * U;
#pragma unroll
    for (int m = 0; m < U; ++m) pk[m] = live ? __ldcg(b2 + m) : make_double2(0.0, 0.0);
    for (int k = 1; k < (live ? ns : 1); ++k) {
#pragma unroll
      for (int m = 0; m < U; ++m) {
        const double2 v2 = __ldcg(b2 + (size_t)k * (W::NV / 2) + m);
        pk[m].x += v2.x;
        pk[m].y += v2.y;
      }
    }
    const double sc = pt.inv_n(f);
#pragma unroll
    for (int m = 0; m < U; ++m) {
      if (!live) break;
      pk[m].x *= sc;
      pk[m].y *= sc;
      bad |= !isfinite(pk[m].x) || !isfinite(pk[m].y);
      const int u = q * U + m;  // 16-byte unit of V_i
      if (u < I / 2) {
        sV[i][2 * u * (I + 1)] = mk(pk[m].x, 0.0);
        sV[i][(2 * u + 1) * (I + 1)] = mk(pk[m].y, 0.0);
      } else {  // the lower entry V_cr = conj(V_rc) goes to the factor's place
        int r, c;
        upper_decode<I>(u - I / 2, r, c);
        sV[i][c * I + r] = mk(pk[m].x, -pk[m].y);
      }
    }
  } else {
    // one packed value per lane (I^3 <= 32)
    static_assert(W::NV <= 32, "one value per lane");
    if (lane < W::NV) {
      double v = __ldcg(slots + lane);
      for (int k = 1; k < ns; ++k) v += __ldcg(slots + (size_t)k * W::NV + lane);
      v *= pt.inv_n(f);
      bad = !isfinite(v);
      const int vi = lane / (I * I), m = lane % (I * I);
      if (m < I) {
        sV[vi][m * (I + 1)] = mk(v, 0.0);
      } else {
        int r, c;
        upper_decode<I>((m - I) / 2, r, c);
        if ((m - I) % 2 == 0) sV[vi][c * I + r].re = v;
        else sV[vi][c * I + r].im = -v;
      }
    }
  }
  if (bad) raise_status(a.status, kDevNonfinite, f);
  if (a.lam_next && live) {  // commit the new Lambda (computed during pass B)
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int m = 0; m < JL; ++m) {
      const int j = q + Q * m;
      if (j < J) {
        a.lam[(size_t)f * J * I + j * I + i] = lnext[m];
        ta->set_lam(j, i, (T)lnext[m]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int r = q + Q * m;
    if (live && r < I) sX[i][r] = xr[m];
  }
  __syncwarp();
  const bool ok = wide_ldl<I>(sV, sL, sRd, i, q);

  // K sweeps from the one factorisation: p_i = V_i^{-1} [P^{-H}]_i
  bool sing_mid = false;
  for (int sweep = 0; sweep < a.K; ++sweep) {
    wide_solve<I>(sV, sRd, sX, i, q);
    if (sweep + 1 < a.K) {  // P^{-H} of the intermediate P
      cpx<double> t[R];
      sing_mid |= !(pinvh_wide<I>(sX, i, q, t) > 0.0);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + Q * m;
        if (live && r < I) sX[i][r] = t[m];
      }
      __syncwarp();
    }
  }
  if (live) {  // the new P: rows q + Q m of column i
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + Q * m;
      if (r < I) {
        const cpx<double> pv = sX[i][r];
        reinterpret_cast<double2*>(a.P)[(size_t)f * I * I + r * I + i] = make_double2(pv.re, pv.im);
        ta->set_p(r, i, (T)pv.re, (T)pv.im);
      }
    }
  }
  // the next step's P^{-H} and ln|det P|^2 of the new P (Eq. L2)
  cpx<double> ph[R];
  const double det2 = pinvh_wide<I>(sX, i, q, ph);
  if (live) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + Q * m;
      if (r < I)
        reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I * I + r * I + i] = make_double2(ph[m].re, ph[m].im);
    }
  }
  const bool singular = __any_sync(0xffffffffu, !ok || sing_mid) || !(det2 > 0.0);
  if (lane == 0) {
    if (singular) raise_status(a.status, kDevSingular, f);
    atomicAdd(a.ops, p_update_inversions(a, I));
    a.logdet[f] = log(det2);
  }
}

// k_prep_wide: what k_prep_gj computes (ln|det P|^2, P^{-H} and the pass-A
// table of the current P and Lambda), one warp per problem, with the
// P^{-H} routine of k_psolve_wide (the bits of pinvh_from_columns).
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_prep_wide(FastArgs a) {
  using W = WideP<I>;
  constexpr int Q = W::Q, R = W::R;
  __shared__ cpx<double> sX[I][W::XS];
  const int f = blockIdx.x;
  if (f >= a.F) return;
  const int lane = threadIdx.x;
  const int i = lane % I, q = lane / I;
  const bool live = q < Q;
  ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int r = q + Q * m;
    if (live && r < I) {
      const double2 u = reinterpret_cast<const double2*>(a.P)[(size_t)f * I * I + r * I + i];
      sX[i][r] = mk(u.x, u.y);
      ta->set_p(r, i, (T)u.x, (T)u.y);
    }
  }
  for (int e = lane; e < J * I; e += 32) ta->set_lam(e / I, e % I, (T)a.lam[(size_t)f * J * I + e]);
  __syncwarp();
  cpx<double> ph[R];
  const double det2 = pinvh_wide<I>(sX, i, q, ph);
  if (a.pinvH && live) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + Q * m;
      if (r < I)
        reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I * I + r * I + i] = make_double2(ph[m].re, ph[m].im);
    }
  }
  if (lane == 0) {
    if (!(det2 > 0.0)) raise_status(a.status, kDevSingular, f);
    a.logdet[f] = log(det2);
  }
}

}  // namespace ffca
