// The normal EM update of P (Sec. 4.6 names it as an alternative to the
// fixed-point iteration of Eq. FPI), per problem after pass A in its EM form
// (k_estep<..., EM = true>), which streams y and v once per iteration: there
// is no pass B.
//
// Complete data: the source images x_j of Eq. fullrank, x_j ~ CN(0, v_j
// P^{-H} Lambda_j P^{-1}) (Eq. diagconst).  Over P the expected complete-data
// log-likelihood is J N ln|det P|^2 - sum_i p_i^H W_i p_i with
//     W_i = sum_{n,j} E[x_j x_j^H | y] / (v_j^new lambda_ji^new)
//         = P^{-H} Omega_i P^{-1},   Omega_i = sum_j T_j / lambda_ji^new,
//     T_j = sum_n (mu~_j mu~_j^H + diag phi~_j) / v_j^new
// (posterior of the entering state, Eqs. mutilde0 / Phitilde0; the new v and
// Lambda of Eqs. updatev / Lambdaupdate).  Its stationarity condition has
// Eq. FPI's form with V_i replaced by W_i / (J N); K sweeps of that map from
// the entering P (all columns from one P_k^{-H} per sweep):
//     p_i <- (W_i / (J N))^{-1} [P_k^{-H}]_i = J N P Omega_i^{-1} P^H [P_k^{-H}]_i,
// which for the first sweep (P_0 = P) is J N P Omega_i^{-1} e_i: no inverse
// of P is needed to form it.  Pass A gives the diagonal of T_j as the
// Lambda sums (T_j[a][a] = N lambda_ja^new) and its off-diagonal entries as
// T_j[a][b] = I lambda_ja lambda_jb sum_n u_j z_a conj(z_b) (old Lambda).
//
//   k_psolve_em  one warp per 32 / I problems, lane (g, i) owning column i
//                of problem g (I = 8: the entering P and both Lambdas in the
//                problem's shared record, not in registers): the slot sums
//                (the whole warp, through shared memory), the new Lambda and
//                the problem's L2 of the
//                entering state (the work pass B's producer does in the
//                fixed-point iteration), Omega_i = L D L^H, the K sweeps, then
//                P^{-H} and ln|det P|^2 of the new P; with a trace, the last
//                block to finish sums the problems' L2.
#pragma once

#include "ffca_big.cuh"
#include "ffca_psolve_wide.cuh"

namespace ffca {

template <int I, int J>
struct EmShape {
  static constexpr int NA = J * I;                 // Lambda sums (as pass A)
  static constexpr int NPAIR = I * (I - 1) / 2;    // entries a < b of T_j
  static constexpr int NV = NA + 2 + 2 * J * NPAIR;  // + the two L2 sums, + (re, im) per j and pair
  static constexpr int G = 32 / I;                 // problems per warp
  static constexpr int NL = NPAIR > 0 ? NPAIR : 1; // storage of the strictly lower entries
  // I > 4: the entering P and both Lambdas of each problem in shared memory
  // (as registers they would take more than a lane holds)
  static constexpr bool BIG = I > 4;
  static constexpr int PSM = BIG ? G * (I * I * 2 + 2 * J * I) : 0;  // doubles
  // I > 4 with K > 1: each lane's L D L^H factor of Omega_i, kept in shared
  // memory between the sweeps (held in registers across the sweep loop it
  // would not fit)
  static constexpr int FAC = BIG ? 2 * NL + I : 0;  // doubles per lane
  static constexpr int SMEM =
      BigLane<I>::SMEM + G * NV * (int)sizeof(double) + PSM * (int)sizeof(double) + 32 * FAC * (int)sizeof(double);
};

template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_psolve_em(FastArgs a) {
  using ES = EmShape<I, J>;
  constexpr int G = ES::G;
  constexpr int NV = ES::NV, NA = ES::NA, NPAIR = ES::NPAIR;
  extern __shared__ __align__(16) unsigned char em_smem[];
  const int lane = threadIdx.x;
  const int g = lane / I, i = lane % I;
  const int f0 = blockIdx.x * G + g;
  const bool active = g < G && f0 < a.F;
  const int f = active ? f0 : 0;  // idle lanes shadow problem 0 and write nothing
  cpx<double>* M = reinterpret_cast<cpx<double>*>(em_smem) + (size_t)(g < G ? g : G) * I * BigLane<I>::LDM;
  double* sums = reinterpret_cast<double*>(em_smem + BigLane<I>::SMEM);  // [G][NV]
  const Partition pt = a.part;

  // the slot sums of the block's problems (slot order), spread over the
  // whole warp: lane l takes the values l + 32 c of the flattened [G][NV]
  // sums and issues its loads of one slot together
  constexpr int PER = (G * NV + 31) / 32;
  if constexpr (PER <= 16) {
    const double* src[PER];
    int ns[PER];
    double acc[PER];
    int nsmax = 0;
#pragma unroll
    for (int c = 0; c < PER; ++c) {
      const int x = lane + 32 * c;
      const int ff = blockIdx.x * G + x / NV;
      const bool ok = x < G * NV && ff < a.F;
      ns[c] = ok ? pt.nslots(ff) : 0;
      src[c] = a.part_buf + ((size_t)(ok ? ff : 0) * pt.max_slots) * NV + x % NV;
      acc[c] = 0.0;
      nsmax = max(nsmax, ns[c]);
    }
    for (int k = 0; k < nsmax; ++k)
#pragma unroll
      for (int c = 0; c < PER; ++c)
        if (k < ns[c]) acc[c] += __ldcg(src[c] + (size_t)k * NV);
#pragma unroll
    for (int c = 0; c < PER; ++c)
      if (lane + 32 * c < G * NV) sums[lane + 32 * c] = acc[c];
  } else {  // I > 4: eight values of a lane at a time
    constexpr int CH = 8;
#pragma unroll 1
    for (int c0 = 0; c0 < PER; c0 += CH) {
      const double* src[CH];
      int ns[CH];
      double acc[CH];
      int nsmax = 0;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int x = lane + 32 * (c0 + c);
        const int ff = blockIdx.x * G + x / NV;
        const bool ok = c0 + c < PER && x < G * NV && ff < a.F;
        ns[c] = ok ? pt.nslots(ff) : 0;
        src[c] = a.part_buf + ((size_t)(ok ? ff : 0) * pt.max_slots) * NV + (ok ? x % NV : 0);
        acc[c] = 0.0;
        nsmax = max(nsmax, ns[c]);
      }
      for (int k = 0; k < nsmax; ++k)
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (k < ns[c]) acc[c] += __ldcg(src[c] + (size_t)k * NV);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int x = lane + 32 * (c0 + c);
        if (c0 + c < PER && x < G * NV) sums[x] = acc[c];
      }
    }
  }
  // the entering P (all columns) and Lambda of this lane's problem: in
  // registers for I <= 4, else in the problem's shared record (each lane
  // loads its column)
  constexpr bool BIG = ES::BIG;
  constexpr int RP = BIG ? 1 : I, RJ = BIG ? 1 : J;
  constexpr int REC = I * I * 2 + 2 * J * I;  // doubles of a problem's record: P, old Lambda, new Lambda
  double* rec = reinterpret_cast<double*>(em_smem + BigLane<I>::SMEM + G * NV * sizeof(double)) +
                (size_t)(g < G ? g : 0) * REC;
  cpx<double> P0r[RP][RP];
  double lold_r[RJ][RP], lnew_r[RJ][RP];
  if constexpr (BIG) {
    if (g < G) {
#pragma unroll
      for (int r = 0; r < I; ++r) {
        const double2 q = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I * I + r * I + i);
        rec[2 * (r * I + i)] = q.x;
        rec[2 * (r * I + i) + 1] = q.y;
      }
#pragma unroll
      for (int j = 0; j < J; ++j) rec[2 * I * I + j * I + i] = __ldcg(a.lam + (size_t)f * J * I + j * I + i);
    }
  } else {
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) {
        const double2 q = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I * I + r * I + c);
        P0r[r][c] = mk(q.x, q.y);
      }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int c = 0; c < I; ++c) lold_r[j][c] = __ldcg(a.lam + (size_t)f * J * I + j * I + c);
  }
  auto P0 = [&](int r, int c) -> cpx<double> {
    if constexpr (BIG) return mk(rec[2 * (r * I + c)], rec[2 * (r * I + c) + 1]);
    else return P0r[r][c];
  };
  auto LOLD = [&](int j, int c) -> double {
    if constexpr (BIG) return rec[2 * I * I + j * I + c]; else return lold_r[j][c];
  };
  auto LNEW = [&](int j, int c) -> double {
    if constexpr (BIG) return rec[2 * I * I + J * I + j * I + c]; else return lnew_r[j][c];
  };
  const double logdet_old = __ldcg(a.logdet + f);
  __syncwarp();  // sums complete; every lane has read P and Lambda before any lane writes them
  const double* tot = sums + (size_t)(g < G ? g : 0) * NV;
  const int n = pt.frames(f);
  const double nd = (double)n;

  // the new Lambda (Eq. Lambdaupdate: lambda_ja I sum_n t_ja / s_j / N)
  bool bad = false;
  if constexpr (BIG) {  // column i by this lane
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const double l = LOLD(j, i) * ((double)I * pt.inv_n(f)) * tot[j * I + i];
      bad |= !(l > 0.0) || !isfinite(l);
      if (g < G) rec[2 * I * I + J * I + j * I + i] = l;
    }
    __syncwarp();
  } else {
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int c = 0; c < I; ++c) {
        lnew_r[j][c] = LOLD(j, c) * ((double)I * pt.inv_n(f)) * tot[j * I + c];
        bad |= !(lnew_r[j][c] > 0.0) || !isfinite(lnew_r[j][c]);
      }
  }
  // L2 of the entering state (Eq. L2)
  const double lf = -(double)I * nd * kLnPi + nd * logdet_old - tot[NA] - 0.69314718055994530942 * tot[NA + 1];
  bad |= !isfinite(lf);

  // Omega_i: diagonal sum_j N lambda_ja^new / lambda_ji^new; above it
  // sum_j I lambda_ja lambda_jb S_j[a][b] / lambda_ji^new (old Lambda in the
  // products, S_j the pass-A sums); kept as the real diagonal and the
  // strictly lower entries Omega_ba = conj(Omega_ab)
  double rl[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    double lji;
    if constexpr (BIG) {
      lji = LNEW(j, i);
    } else {
      lji = LNEW(j, 0);
#pragma unroll
      for (int c = 1; c < I; ++c)
        if (c == i) lji = LNEW(j, c);
    }
    rl[j] = 1.0 / lji;
  }
  // Omega_i's diagonal entry c (formed again for the pivot check: I > 4
  // keeps no copy in registers)
  auto omega_diag = [&](int c) -> double {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < J; ++j) s = fma(nd * LNEW(j, c), rl[j], s);
    return s;
  };
  double dv[I], d0[BIG ? 1 : I], rd[I];
  cpx<double> lo[ES::NL];
#pragma unroll
  for (int c = 0; c < I; ++c) {
    dv[c] = omega_diag(c);
    if constexpr (!BIG) d0[c] = dv[c];
  }
  {
    int pq = 0;
#pragma unroll
    for (int aa = 0; aa < I; ++aa)
#pragma unroll
      for (int bb = aa + 1; bb < I; ++bb, ++pq) {
        cpx<double> s = mk(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const double w = (double)I * LOLD(j, aa) * LOLD(j, bb) * rl[j];
          const double* t = tot + NA + 2 + 2 * (j * NPAIR + pq);
          s.re = fma(w, t[0], s.re);
          s.im = fma(w, t[1], s.im);
        }
        lo[lo_index(bb, aa)] = cconj(s);
      }
  }
  bool singular = false;
#pragma unroll
  for (int c = 0; c < I; ++c) bad |= !isfinite(dv[c]);
#pragma unroll
  for (int c = 0; c < NPAIR; ++c) bad |= !isfinite(lo[c].re) || !isfinite(lo[c].im);
  if constexpr (I == 1) {
    singular = !(dv[0] > 0.0) || !isfinite(dv[0]);
    rd[0] = 1.0 / dv[0];
  } else {
    singular = !ldl_factor<I>(dv, lo, rd);
#pragma unroll
    for (int c = 0; c < I; ++c) {  // dv holds the pivots D
      if constexpr (BIG) singular |= !(dv[c] > kCholRtol * omega_diag(c));
      else singular |= !(dv[c] > kCholRtol * d0[c]);
    }
  }

  // commit the new Lambda (column i of the problem's Lambda entries)
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      double l;
      if constexpr (BIG) {
        l = LNEW(j, i);
      } else {
        l = LNEW(j, 0);
#pragma unroll
        for (int c = 1; c < I; ++c)
          if (c == i) l = LNEW(j, c);
      }
      a.lam[(size_t)f * J * I + j * I + i] = l;
      ta->set_lam(j, i, (T)l);
    }
    if (i == 0) a.llf[f] = lf;
    if (bad) raise_status(a.status, kDevNonfinite, f);
  }

  // K sweeps; col holds column i of the current P.  The first (x = P^H
  // P^{-H} e_i = e_i) is written out before the loop of the later ones, so
  // that K = 1 runs none of the loop's register traffic (at I = 8 the loop
  // state does not fit the registers).
  const double jn = (double)J * nd;
  cpx<double> col[I];
  auto sweep_tail = [&](cpx<double> (&x)[I]) {  // col = J N P Omega_i^{-1} x
    if constexpr (I == 1) {
      x[0] = cscale(x[0], rd[0]);
    } else {
      ldl_solve<I>(lo, rd, x);
    }
#pragma unroll
    for (int r = 0; r < I; ++r) {
      cpx<double> s = mk(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < I; ++c) cfma(s, P0(r, c), x[c]);
      col[r] = cscale(s, jn);
    }
  };
  {
    cpx<double> x[I];
#pragma unroll
    for (int r = 0; r < I; ++r) x[r] = mk(r == i ? 1.0 : 0.0, 0.0);
    sweep_tail(x);
  }
  double* fac = reinterpret_cast<double*>(em_smem + BigLane<I>::SMEM + G * NV * sizeof(double) +
                                          ES::PSM * sizeof(double)) + (size_t)lane * ES::FAC;
  if constexpr (BIG) {
    if (a.K > 1) {
#pragma unroll
      for (int c = 0; c < ES::NL; ++c) {
        fac[2 * c] = lo[c].re;
        fac[2 * c + 1] = lo[c].im;
      }
#pragma unroll
      for (int c = 0; c < I; ++c) fac[2 * ES::NL + c] = rd[c];
    }
  }
  for (int sweep = 1; sweep < a.K; ++sweep) {
    cpx<double> q[I];  // column i of the current P's P^{-H}
#pragma unroll
    for (int r = 0; r < I; ++r) q[r] = col[r];
    pinvh_from_columns<I>(q, M, g, i, singular);
    cpx<double> x[I];
#pragma unroll
    for (int c = 0; c < I; ++c) {  // x = P^H q with the entering P
      cpx<double> s = mk(0.0, 0.0);
#pragma unroll
      for (int r = 0; r < I; ++r) cfmac(s, P0(r, c), q[r]);
      x[c] = s;
    }
    if constexpr (BIG) {  // the factor back from shared memory
      cpx<double> lo2[ES::NL];
      double rd2[I];
#pragma unroll
      for (int c = 0; c < ES::NL; ++c) lo2[c] = mk(fac[2 * c], fac[2 * c + 1]);
#pragma unroll
      for (int c = 0; c < I; ++c) rd2[c] = fac[2 * ES::NL + c];
      ldl_solve<I>(lo2, rd2, x);
#pragma unroll
      for (int r = 0; r < I; ++r) {
        cpx<double> s = mk(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < I; ++c) cfma(s, P0(r, c), x[c]);
        col[r] = cscale(s, jn);
      }
    } else {
      sweep_tail(x);
    }
  }
  if (active) {
    ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
#pragma unroll
    for (int r = 0; r < I; ++r) {
      reinterpret_cast<double2*>(a.P)[(size_t)f * I * I + r * I + i] = make_double2(col[r].re, col[r].im);
      ta->set_p(r, i, (T)col[r].re, (T)col[r].im);
    }
  }
  // P^{-H} and ln|det P|^2 of the new P (the next iteration's L2 needs it)
  const double det2 = pinvh_from_columns<I>(col, M, g, i, singular);
  if (active) {
#pragma unroll
    for (int r = 0; r < I; ++r)
      reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I * I + r * I + i] = make_double2(col[r].re, col[r].im);
    if (singular) raise_status(a.status, kDevSingular, f);
    if (i == 0) {
      atomicAdd(a.ops, p_update_inversions(a, I));
      a.logdet[f] = log(det2);
    }
  }
  // with a trace: the last block to finish sums the problems' L2
  if (a.trace) {
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
      last = atomicAdd(a.gcnt, 1u) == gridDim.x - 1;
      if (last) *a.gcnt = 0u;  // ready for the next launch
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      finalize_trace(a);
    }
  }
}

// k_psolve_em_wide: the EM step above for I = 3 or 8 with one warp per
// problem (lane (i, q) as in k_psolve_wide), for a few hundred problems,
// where the packed form leaves most FP64 units idle: the slot sums, the new
// Lambda and the entering state's L2 spread over the warp; Omega_i formed
// entry by entry into shared memory and factored by wide_ldl; the sweeps by
// wide_solve and the products with the entering P by rows; P^{-H} and
// ln|det P|^2 by pinvh_wide (the bits of pinvh_from_columns).  With a
// trace the last block to finish sums the problems' L2.
template <typename T, int I, int J>
__global__ void __launch_bounds__(32) k_psolve_em_wide(FastArgs a) {
  using W = WideP<I>;
  using ES = EmShape<I, J>;
  constexpr int Q = W::Q, R = W::R;
  constexpr int NV = ES::NV, NA = ES::NA, NPAIR = ES::NPAIR;
  constexpr int NTRI = I * (I + 1) / 2;  // entries of a lower triangle with its diagonal
  __shared__ cpx<double> sV[I][W::VS];   // Omega_i, then its factor
  __shared__ cpx<double> sX[I][W::XS];   // x_i, then column i of the new P
  __shared__ cpx<double> sL[I][W::XS];   // factorisation scratch, then P^{-H} columns
  __shared__ double sRd[I][W::XS];
  __shared__ double sSum[NV];            // the problem's slot sums
  __shared__ cpx<double> sP0[I][I];      // the entering P
  __shared__ double sLold[J][I], sLnew[J][I], sRl[I][J];  // Lambda old and new, 1 / lambda_ji^new
  const int f = blockIdx.x;
  if (f >= a.F) return;
  const int lane = threadIdx.x;
  const int i = lane % I, q = lane / I;
  const bool live = q < Q;
  const Partition pt = a.part;

  // the slot sums (slot order), the entering P and Lambda
  {
    const int ns = pt.nslots(f);
    const double* base = a.part_buf + (size_t)f * pt.max_slots * NV;
    for (int x = lane; x < NV; x += 32) {
      double acc = __ldcg(base + x);
      for (int k = 1; k < ns; ++k) acc += __ldcg(base + (size_t)k * NV + x);
      sSum[x] = acc;
    }
    for (int e = lane; e < I * I; e += 32) {
      const double2 u = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I * I + e);
      sP0[e / I][e % I] = mk(u.x, u.y);
    }
    for (int e = lane; e < J * I; e += 32) sLold[e / I][e % I] = __ldcg(a.lam + (size_t)f * J * I + e);
  }
  const double logdet_old = __ldcg(a.logdet + f);
  const double nd = (double)pt.frames(f);
  __syncwarp();

  // the new Lambda (Eq. Lambdaupdate) and the entering state's L2 (Eq. L2)
  bool bad = false;
  ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, f);
  for (int e = lane; e < J * I; e += 32) {
    const int j = e / I, c = e % I;
    const double l = sLold[j][c] * ((double)I * pt.inv_n(f)) * sSum[j * I + c];
    bad |= !(l > 0.0) || !isfinite(l);
    sLnew[j][c] = l;
    a.lam[(size_t)f * J * I + e] = l;
    ta->set_lam(j, c, (T)l);
  }
  {
    const double lf = -(double)I * nd * kLnPi + nd * logdet_old - sSum[NA] - 0.69314718055994530942 * sSum[NA + 1];
    bad |= !isfinite(lf);
    if (lane == 0) a.llf[f] = lf;
  }
  __syncwarp();
  for (int e = lane; e < J * I; e += 32) sRl[e % I][e / I] = 1.0 / sLnew[e / I][e % I];
  __syncwarp();

  // Omega_i: diagonal sum_j N lambda_jc^new / lambda_ji^new; below it
  // conj(sum_j I lambda_ja lambda_jb S_j[a][b] / lambda_ji^new), a < b (old
  // Lambda in the products, S_j the pass-A sums)
  for (int e = lane; e < I * NTRI; e += 32) {
    const int ii = e / NTRI;
    int rr, cc;
    tri_decode(e % NTRI, rr, cc);
    cpx<double> o;
    if (rr == cc) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < J; ++j) s = fma(nd * sLnew[j][cc], sRl[ii][j], s);
      o = mk(s, 0.0);
    } else {
      const int aa = cc, bb = rr;
      const int pq = aa * (2 * I - aa - 1) / 2 + (bb - aa - 1);  // pair (aa, bb) in row order
      cpx<double> s = mk(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const double w = (double)I * sLold[j][aa] * sLold[j][bb] * sRl[ii][j];
        const double* t = sSum + NA + 2 + 2 * (j * NPAIR + pq);
        s.re = fma(w, t[0], s.re);
        s.im = fma(w, t[1], s.im);
      }
      o = cconj(s);
    }
    bad |= !isfinite(o.re) || !isfinite(o.im);
    sV[ii][rr * I + cc] = o;
  }
  if (bad) raise_status(a.status, kDevNonfinite, f);
  __syncwarp();
  const bool ok = wide_ldl<I>(sV, sL, sRd, i, q);

  // K sweeps; the first from x_i = P^H P^{-H} e_i = e_i
  const double jn = (double)J * nd;
  bool sing_mid = false;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int r = q + Q * m;
    if (live && r < I) sX[i][r] = mk(r == i ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  for (int sweep = 0; sweep < a.K; ++sweep) {
    if (sweep > 0) {  // x_i = P^H [P_k^{-H}]_i with the entering P
      cpx<double> t[R];
      sing_mid |= !(pinvh_wide<I>(sX, i, q, t) > 0.0);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + Q * m;
        if (live && r < I) sL[i][r] = t[m];
      }
      __syncwarp();
      cpx<double> xr[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int c = q + Q * m;
        cpx<double> s = mk(0.0, 0.0);
        if (live && c < I) {
#pragma unroll
          for (int r = 0; r < I; ++r) cfmac(s, sP0[r][c], sL[i][r]);
        }
        xr[m] = s;
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int c = q + Q * m;
        if (live && c < I) sX[i][c] = xr[m];
      }
      __syncwarp();
    }
    wide_solve<I>(sV, sRd, sX, i, q);
    cpx<double> cr[R];  // column i of the new P: J N P Omega_i^{-1} x_i
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + Q * m;
      cpx<double> s = mk(0.0, 0.0);
      if (live && r < I) {
#pragma unroll
        for (int c = 0; c < I; ++c) cfma(s, sP0[r][c], sX[i][c]);
      }
      cr[m] = cscale(s, jn);
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + Q * m;
      if (live && r < I) sX[i][r] = cr[m];
    }
    __syncwarp();
  }
  if (live) {  // the new P: rows q + Q m of column i
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
  // P^{-H} and ln|det P|^2 of the new P (the next iteration's L2 needs it)
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
  // with a trace: the last block to finish sums the problems' L2
  if (a.trace) {
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
      last = atomicAdd(a.gcnt, 1u) == gridDim.x - 1;
      if (last) *a.gcnt = 0u;  // ready for the next launch
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      finalize_trace(a);
    }
  }
}

}  // namespace ffca
