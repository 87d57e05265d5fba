// The P step of Eq. FPI for eight microphones with one warp per problem.
//
// An FP64 warp instruction occupies its SM sub-partition's FP64 unit for 64
// cycles on this part (2 FP64 FMAs per clock per SM, 4 sub-partitions), with
// any number of active lanes.  The lane-per-column form (k_psolve_ldl: four
// problems per warp, each lane factoring and solving its own 8 x 8 V_i)
// issues about 1500 FP64 instructions per warp on 130 warps for 513
// problems: one warp per SM, three of every four sub-partitions idle.  Here
// each problem has a warp of its own, lane (i, q) = (lane % 8, lane / 8),
// and the work inside each matrix is spread over the lanes:
//
//   L D L^H of V_i   the four lanes q of V_i share the entries of each
//                    step's trailing triangle (row-major order, entry
//                    q + 4 m); the matrices live in shared memory;
//   the solves       V_i p_i = [P^{-H}]_i, rows of each substitution step
//                    over the four lanes;
//   P^{-H}           Gauss-Jordan with partial pivoting on P^H, lane (c, h)
//                    holding rows h and h + 4 of column c (gj_inverse_wide):
//                    every entry takes the same operations, in the same
//                    order, as in gj_inverse_cols (the routine that k_prep_gj
//                    and the other P updates use), so the P^{-H} carried to
//                    the next step has the same bits as the one recomputed
//                    from P at the start of a call.
//
// So a warp issues about a third of the FP64 instructions of the
// lane-per-column form, and the 513 warps of a 513-problem step use every
// sub-partition of the GPU.
#pragma once

#include "ffca_big.cuh"

namespace ffca {

template <int I>
struct WideP {
  static_assert(I == 8, "the wide P step is laid out for I = 8");
  static constexpr int Q = 32 / I;         // lanes per matrix
  static constexpr int VS = I * I + 1;     // stride of one V_i (complex entries; the pad skews the banks)
  static constexpr int XS = I + 1;         // stride of one vector
  static constexpr int NV = I * I * I;     // values per slot of pass B's partial sums
  static constexpr int PAIRS = I * (I - 1) / 2;
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
template <int I>
__device__ inline void upper_decode(int p, int& r, int& c) {
  r = 0;
  while (p >= I - 1 - r) {
    p -= I - 1 - r;
    ++r;
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

// P^{-H} of the P whose column i is sX[i][0 .. 7], and |det P|^2: lane
// (c, h) gathers rows h, h + 4 of column c of P^H (conj(P[c][r])), inverts,
// and leaves (P^{-H})[h][c], [h + 4][c] in q0, q1.
__device__ inline double pinvh_wide8(const cpx<double> (*sX)[WideP<8>::XS], int c, int h, cpx<double>& q0,
                                     cpx<double>& q1) {
  q0 = cconj(sX[h][c]);
  q1 = cconj(sX[h + 4][c]);
  return gj_inverse_wide8(q0, q1, c, h);
}

// k_psolve_wide: one P step of Eq. FPI (K sweeps) for I = 8, one warp per
// problem (blocks of 32 threads; with a trace the last block sums it).  The
// outputs are those of k_psolve_ldl: the new Lambda committed, P and its
// pass-A table, P^{-H}, ln|det P|^2, the inversion count and the status.
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_psolve_wide(FastArgs a) {
  using W = WideP<I>;
  constexpr int Q = W::Q;
  __shared__ cpx<double> sV[I][W::VS];   // V_i, then its unit lower factor L_i (row-major, lower part)
  __shared__ cpx<double> sX[I][W::XS];   // column i of P^{-H}, then p_i
  __shared__ cpx<double> sL[I][W::XS];   // scaled column k of the factorisation step
  __shared__ double sRd[I][W::XS];       // 1 / D of L_i D_i L_i^H
  if (trace_block(a)) return;
  const int f = blockIdx.x;
  if (f >= a.F) return;
  const int lane = threadIdx.x;
  const int i = lane % I, q = lane / I;  // matrix / column i, quarter q (as (c, h) in the inverse)
  const Partition pt = a.part;

  // every global load first: the new Lambda, column i of P^{-H} (rows q,
  // q + 4) and a quarter of V_i's slots (eight 16-byte units of each)
  double lnext[(J + Q - 1) / Q];
  if (a.lam_next) {
#pragma unroll
    for (int m = 0; m < (J + Q - 1) / Q; ++m) {
      const int j = q + Q * m;
      lnext[m] = j < J ? __ldcg(a.lam_next + (size_t)f * J * I + j * I + i) : 0.0;
    }
  }
  cpx<double> x0, x1;
  {
    const double2* ph = reinterpret_cast<const double2*>(a.pinvH) + (size_t)f * I * I;
    const double2 u0 = __ldcg(ph + q * I + i), u1 = __ldcg(ph + (q + 4) * I + i);
    x0 = mk(u0.x, u0.y);
    x1 = mk(u1.x, u1.y);
  }
  constexpr int U = I * I / 2 / Q;  // 16-byte units of V_i per lane
  double2 pk[U];
  {
    const int ns = pt.nslots(f);  // >= 1: every problem has a slot
    const double2* b2 =
        reinterpret_cast<const double2*>(a.part_buf + (size_t)f * pt.max_slots * W::NV + i * I * I) + q * U;
#pragma unroll
    for (int m = 0; m < U; ++m) pk[m] = __ldcg(b2 + m);
    for (int k = 1; k < ns; ++k) {
#pragma unroll
      for (int m = 0; m < U; ++m) {
        const double2 v2 = __ldcg(b2 + (size_t)k * (W::NV / 2) + m);
        pk[m].x += v2.x;
        pk[m].y += v2.y;
      }
    }
  }
  if (a.lam_next) {  // commit the new Lambda (computed during pass B)
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int m = 0; m < (J + Q - 1) / Q; ++m) {
      const int j = q + Q * m;
      if (j < J) {
        a.lam[(size_t)f * J * I + j * I + i] = lnext[m];
        ta->set_lam(j, i, (T)lnext[m]);
      }
    }
  }
  sX[i][q] = x0;
  sX[i][q + 4] = x1;
  {
    const double sc = pt.inv_n(f);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < U; ++m) {
      pk[m].x *= sc;
      pk[m].y *= sc;
      bad |= !isfinite(pk[m].x) || !isfinite(pk[m].y);
    }
    if (bad) raise_status(a.status, kDevNonfinite, f);
    // packed Hermitian V_i: I diagonal values, then (re, im) of V_rc, r < c,
    // in row order; the lower entry V_cr = conj(V_rc) goes to the factor's place
#pragma unroll
    for (int m = 0; m < U; ++m) {
      const int u = q * U + m;  // 16-byte unit of V_i
      if (u < I / 2) {
        sV[i][2 * u * (I + 1)] = mk(pk[m].x, 0.0);
        sV[i][(2 * u + 1) * (I + 1)] = mk(pk[m].y, 0.0);
      } else {
        int r, c;
        upper_decode<I>(u - I / 2, r, c);
        sV[i][c * I + r] = mk(pk[m].x, -pk[m].y);
      }
    }
  }
  __syncwarp();
  double d0[I];  // the diagonal before the factorisation
#pragma unroll
  for (int k = 0; k < I; ++k) d0[k] = sV[i][k * (I + 1)].re;

  // L D L^H in place (right-looking, no square roots).  Lane q takes the
  // entries q + 4 m of each step's trailing triangle; their places relative
  // to the triangle's corner are the same at every step (the row-major
  // order of a triangle starts with that of every smaller one).
  constexpr int ME = (I * (I - 1) / 2 + Q - 1) / Q;  // entries per lane at the first step
  int e_rc[ME], e_r[ME], e_c[ME];                   // rr * I + cc, rr * I, cc
#pragma unroll
  for (int m = 0; m < ME; ++m) {
    int rr, cc;
    tri_decode(q + Q * m, rr, cc);
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
      if (r < I) {
        lr[m] = cscale(V[r * I + k], inv);
        sL[i][r] = lr[m];
      }
    }
    if (q == 0) sRd[i][k] = inv;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < (NT + Q - 1) / Q; ++m) {
      if (q + Q * m < NT) {  // V_rc -= V_rk conj(l_c), k < c <= r (the diagonal's real part is |V_rk|^2 / d)
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
      if (r < I) V[r * I + k] = lr[m];
    }
  }
  __syncwarp();
  // K sweeps from the one factorisation: p_i = V_i^{-1} [P^{-H}]_i
  const cpx<double>* L = sV[i];
  bool sing_mid = false;
  for (int sweep = 0; sweep < a.K; ++sweep) {
#pragma unroll
    for (int k = 0; k < I - 1; ++k) {  // L z = x
      const cpx<double> zk = sX[i][k];
      const int NR = I - 1 - k;
#pragma unroll
      for (int m = 0; m < (NR + Q - 1) / Q; ++m) {
        const int r = k + 1 + q + Q * m;
        if (r < I) {
          const cpx<double> l = L[r * I + k];
          cpx<double> v = sX[i][r];
          cfma(v, mk(-l.re, -l.im), zk);
          sX[i][r] = v;
        }
      }
      __syncwarp();
    }
    sX[i][q] = cscale(sX[i][q], sRd[i][q]);
    sX[i][q + 4] = cscale(sX[i][q + 4], sRd[i][q + 4]);
    __syncwarp();
#pragma unroll
    for (int k = I - 1; k > 0; --k) {  // L^H p = z: (L^H)_rk = conj(L_kr)
      const cpx<double> zk = sX[i][k];
#pragma unroll
      for (int m = 0; m < (k + Q - 1) / Q; ++m) {
        const int r = q + Q * m;
        if (r < k) {
          const cpx<double> l = L[k * I + r];
          cpx<double> v = sX[i][r];
          cfma(v, mk(-l.re, l.im), zk);
          sX[i][r] = v;
        }
      }
      __syncwarp();
    }
    if (sweep + 1 < a.K) {  // P^{-H} of the intermediate P
      cpx<double> t0, t1;
      sing_mid |= !(pinvh_wide8(sX, i, q, t0, t1) > 0.0);
      __syncwarp();
      sX[i][q] = t0;
      sX[i][q + 4] = t1;
      __syncwarp();
    }
  }
  {  // the new P: rows q, q + 4 of column i
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int r = q + 4 * m;
      const cpx<double> pv = sX[i][r];
      reinterpret_cast<double2*>(a.P)[(size_t)f * I * I + r * I + i] = make_double2(pv.re, pv.im);
      ta->set_p(r, i, (T)pv.re, (T)pv.im);
    }
  }
  // the next step's P^{-H} and ln|det P|^2 of the new P (Eq. L2)
  cpx<double> q0, q1;
  const double det2 = pinvh_wide8(sX, i, q, q0, q1);
  {
    double2* ph = reinterpret_cast<double2*>(a.pinvH) + (size_t)f * I * I;
    ph[q * I + i] = make_double2(q0.re, q0.im);
    ph[(q + 4) * I + i] = make_double2(q1.re, q1.im);
  }
  const bool singular = __any_sync(0xffffffffu, !ok || sing_mid) || !(det2 > 0.0);
  if (lane == 0) {
    if (singular) raise_status(a.status, kDevSingular, f);
    atomicAdd(a.ops, p_update_inversions(a, I));
    a.logdet[f] = log(det2);
  }
}

}  // namespace ffca
