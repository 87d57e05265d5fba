// Newton's method for P (Sec. 4.6 names it as an alternative to the
// fixed-point iteration of Eq. FPI), per problem after pass B, with the V_i
// of Eq. FPI held fixed (sigma from the new v and Lambda).
//
// Objective, per problem: l(P) = ln|det P|^2 - sum_i p_i^H V_i p_i (L2 / N up
// to terms free of P).  In the 2 I^2 real coordinates of P (direction k is
// E_k = phi_k e_a e_c^T with phi_k = 1 for k < I^2 and i above, k = a I + c
// within each half):
//   gradient  g_k = 2 Re(conj(G_ac) phi_k),  G = P^{-H} - [V_1 p_1 ... V_I p_I]
//   Hessian   H_kl = -2 Re(phi_k phi_l Q_{c_l a_k} Q_{c_k a_l})
//                    - 2 Re(conj(phi_k) phi_l [V_c]_{a_k a_l}) [c_k = c_l = c]
// with Q = P^{-1} (the second differentials of ln det and of the quadratic
// form).  l does not change when a column turns in phase, p_i -> e^{i t} p_i,
// so the step is taken off those I directions: with u_i the unit vector of
// the direction i p_i (supported on column i only, so the u_i are already
// orthogonal), Pi = sum_i u_i u_i^T and Q' = 1 - Pi, the step s solves
// (Q' H Q' - Pi) s = -Q' g and P moves by mu sum_k s_k E_k.  K steps per
// iteration; each inverts P and the 2 I^2 system (two inversions).
//
//   k_psolve_newton  one warp per problem (2 I^2 <= 32: I <= 4), lane l
//                    holding column l of the system (H is symmetric, so also
//                    its row): it builds its column, projects it, and the
//                    warp solves by Gauss-Jordan with partial pivoting on
//                    the lanes' columns (the right-hand side replicated in
//                    every lane); then P^{-H} and ln|det P|^2 of the new P.
#pragma once

#include "ffca_big.cuh"

namespace ffca {

template <typename T, int I>
__global__ void __launch_bounds__(32) k_psolve_newton(FastArgs a) {
  constexpr int I2 = I * I;
  constexpr int n = 2 * I2;  // unknowns
  constexpr int NV = I * I2;  // packed V_i of the slots
  static_assert(n <= 32, "one lane per column: I <= 4");
  __shared__ double sV[NV];              // V_i / N, packed Hermitian per i
  __shared__ cpx<double> sP[I][I];       // the current P
  __shared__ cpx<double> sQ[I][I];       // its inverse
  __shared__ cpx<double> sG[I][I];       // G = P^{-H} - [V_i p_i]
  if (trace_block(a)) return;
  const int lane = threadIdx.x;
  const int f = blockIdx.x;  // one problem per block
  const Partition pt = a.part;

  // commit the new Lambda (computed during pass B) and sum pass B's slots
  const int J = a.J;  // one kernel serves every J
  if (a.lam_next) {
    ParamsARun<T, I> ta(a.tabA, J, f);
    for (int q = lane; q < J * I; q += 32) {
      const double l = __ldcg(a.lam_next + (size_t)f * J * I + q);
      a.lam[(size_t)f * J * I + q] = l;
      ta.set_lam(q / I, q % I, (T)l);
    }
  }
  bool bad = false;
  {
    const int ns = pt.nslots(f);
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV;
    for (int q = lane; q < NV; q += 32) {
      double s = 0.0;
      for (int k = 0; k < ns; ++k) s += __ldcg(base + (size_t)k * NV + q);
      s *= pt.inv_n(f);
      bad |= !isfinite(s);
      sV[q] = s;
    }
  }
  if (lane < I2) {
    const double2 q = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I2 + lane);
    sP[lane / I][lane % I] = mk(q.x, q.y);
  }
  __syncwarp();
  // [V_c]_{r s} from the packed record of c: diagonal, then (re, im) of the
  // entries above it in row order
  auto Vget = [&](int c, int r, int s) -> cpx<double> {
    const double* v = sV + c * I2;
    if (r == s) return mk(v[r], 0.0);
    const int lo = r < s ? r : s, hi = r < s ? s : r;
    const int m = I + 2 * (lo * (2 * I - lo - 1) / 2 + (hi - lo - 1));
    return r < s ? mk(v[m], v[m + 1]) : mk(v[m], -v[m + 1]);
  };

  // this lane's column l = (a_l, c_l, phi_l) of the system (lanes >= n shadow column 0)
  const int l = lane < n ? lane : 0;
  const int al = (l % I2) / I, cl = l % I;
  const bool iml = l >= I2;
  bool singular = false;

  for (int step = 0; step < a.K; ++step) {
    // P^{-1} (cofactors, every lane) and G, one entry per lane
    cpx<double> A[I][I];
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) A[r][c] = sP[r][c];
    {
      cpx<double> C[I][I];
      const cpx<double> det = cofactors<I>(A, C);
      const double d2 = cabs2(det);
      singular |= !(d2 > 0.0) || !isfinite(d2);
      const double inv = 1.0 / d2;
      const cpx<double> rdet = mk(det.re * inv, -det.im * inv);
      if (lane < I2) {
        const int x = lane / I, y = lane % I;
        cpx<double> cyx = C[0][0];
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = 0; c < I; ++c)
            if (r == y && c == x) cyx = C[r][c];
        sQ[x][y] = cmul(cyx, rdet);  // (P^{-1})_{xy} = C_yx / det P
      }
    }
    __syncwarp();
    if (lane < I2) {  // G_ac = conj(Q_ca) - sum_b [V_c]_{ab} P_bc
      const int x = lane / I, c = lane % I;
      cpx<double> s = cconj(sQ[c][x]);
#pragma unroll
      for (int b = 0; b < I; ++b) {
        const cpx<double> t = cmul(Vget(c, x, b), sP[b][c]);
        s = csub(s, t);
      }
      sG[x][c] = s;
    }
    __syncwarp();

    // u_i (unit vectors of the phase turns i p_i) at every coordinate, and at l
    double nrm[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
      double s2 = 0.0;
#pragma unroll
      for (int r = 0; r < I; ++r) s2 += cabs2(A[r][i]);
      nrm[i] = 1.0 / sqrt(s2);
    }
    auto U = [&](int i, int k) -> double {  // compile-time i, k
      const int ak = (k % I2) / I, ck = k % I;
      if (ck != i) return 0.0;
      return (k >= I2 ? A[ak][i].re : -A[ak][i].im) * nrm[i];
    };
    double ul[I];  // u_i[l]
#pragma unroll
    for (int i = 0; i < I; ++i) {
      cpx<double> pai = A[0][i];
#pragma unroll
      for (int r = 1; r < I; ++r)
        if (r == al) pai = A[r][i];
      ul[i] = (cl == i) ? (iml ? pai.re : -pai.im) * nrm[i] : 0.0;
    }

    // column l of H (= row l) and the gradient at every coordinate
    cpx<double> ql[I], qr[I];  // Q_{c_l, a} and Q_{c, a_l} for every a, c
#pragma unroll
    for (int x = 0; x < I; ++x) {
      ql[x] = sQ[cl][x];
      qr[x] = sQ[x][al];
    }
    cpx<double> vl[I];  // [V_{c_l}]_{a, a_l} for every a
#pragma unroll
    for (int x = 0; x < I; ++x) vl[x] = Vget(cl, x, al);
    const cpx<double> phl = iml ? mk(0.0, 1.0) : mk(1.0, 0.0);
    double col[n], g[n];
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const int ak = (k % I2) / I, ck = k % I;
      const cpx<double> phk = k >= I2 ? mk(0.0, 1.0) : mk(1.0, 0.0);
      const cpx<double> t1 = cmul(cmul(phk, phl), cmul(ql[ak], qr[ck]));
      double h = -2.0 * t1.re;
      if (ck == cl) h -= 2.0 * cmul(cmul(cconj(phk), phl), vl[ak]).re;
      col[k] = h;
      const cpx<double> gk = sG[ak][ck];
      g[k] = 2.0 * (k >= I2 ? gk.im : gk.re);
    }
    // projection: with w_i = (H u_i)_l (H symmetric: column l dotted with u_i),
    // W_ki = (H u_i)_k from lane k, S = U^T W:
    // column l of Q' H Q' - Pi = H e_l - U w - W u_l + U S u_l - U u_l
    double w[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) s = fma(col[k], U(i, k), s);
      w[i] = s;
    }
    double S[I][I], Ug[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < n; ++k) t = fma(U(i, k), g[k], t);
      Ug[i] = t;
#pragma unroll
      for (int j = 0; j < I; ++j) S[i][j] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < n; ++k) {  // S = U^T W, row k of W from lane k
#pragma unroll
      for (int j = 0; j < I; ++j) {
        const double wkj = __shfl_sync(0xffffffffu, w[j], k);
#pragma unroll
        for (int i = 0; i < I; ++i) S[i][j] = fma(U(i, k), wkj, S[i][j]);
      }
    }
    double su[I];  // (S u_l)_i - u_i[l]
#pragma unroll
    for (int i = 0; i < I; ++i) {
      double t = -ul[i];
#pragma unroll
      for (int j = 0; j < I; ++j) t = fma(S[i][j], ul[j], t);
      su[i] = t;
    }
    double rhs[n];
#pragma unroll
    for (int k = 0; k < n; ++k) {
      double t = col[k], r = g[k];
#pragma unroll
      for (int j = 0; j < I; ++j) {
        const double wkj = __shfl_sync(0xffffffffu, w[j], k);
        t = fma(-wkj, ul[j], t);          // - W u_l
        t = fma(-U(j, k), w[j], t);       // - U w_l
        t = fma(U(j, k), su[j], t);       // + U (S u_l - u_l)
        r = fma(-U(j, k), Ug[j], r);      // Q' g
      }
      col[k] = lane < n ? t : 0.0;
      rhs[k] = -r;
    }

    // Gauss-Jordan on the lanes' columns with partial pivoting; every lane
    // applies the row operations to its copy of the right-hand side
#pragma unroll
    for (int k = 0; k < n; ++k) {
      int p = k;
      if (lane == k) {
        unsigned long long best = (unsigned long long)__double_as_longlong(col[k]) & 0x7fffffffffffffffull;
#pragma unroll
        for (int r = k + 1; r < n; ++r) {
          const unsigned long long m = (unsigned long long)__double_as_longlong(col[r]) & 0x7fffffffffffffffull;
          if (m > best) {
            best = m;
            p = r;
          }
        }
      }
      p = __shfl_sync(0xffffffffu, p, k);
#pragma unroll
      for (int r = k + 1; r < n; ++r) {
        if (r == p) {
          const double t = col[k];
          col[k] = col[r];
          col[r] = t;
          const double u = rhs[k];
          rhs[k] = rhs[r];
          rhs[r] = u;
        }
      }
      const double piv = __shfl_sync(0xffffffffu, col[k], k);
      singular |= !(piv != 0.0) || !isfinite(piv);
      const double rp = 1.0 / piv;
      const double tk = col[k] * rp, rk = rhs[k] * rp;
#pragma unroll
      for (int r = 0; r < n; ++r) {
        if (r == k) continue;
        const double pc = __shfl_sync(0xffffffffu, col[r], k);
        col[r] = fma(-pc, tk, col[r]);
        rhs[r] = fma(-pc, rk, rhs[r]);
      }
      col[k] = tk;
      rhs[k] = rk;
    }
    // P += mu sum_k s_k E_k (every lane holds s = rhs)
    __syncwarp();
    if (lane < I2) {
      const int x = lane / I, c = lane % I;
      double sr = rhs[0], si = rhs[I2];
#pragma unroll
      for (int k = 1; k < I2; ++k)
        if (k == lane) {
          sr = rhs[k];
          si = rhs[I2 + k];
        }
      sP[x][c] = mk(sP[x][c].re + a.mu * sr, sP[x][c].im + a.mu * si);
    }
    __syncwarp();
  }

  // write the new P (and the pass-A table), its P^{-H} and ln|det P|^2
  cpx<double> A[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) A[r][c] = sP[r][c];
  cpx<double> C[I][I];
  const cpx<double> det = cofactors<I>(A, C);
  const double d2 = cabs2(det);
  singular |= !(d2 > 0.0) || !isfinite(d2);
  if (lane < I2) {
    const int x = lane / I, c = lane % I;
    const cpx<double> pxc = sP[x][c];
    reinterpret_cast<double2*>(a.P)[(size_t)f * I2 + lane] = make_double2(pxc.re, pxc.im);
    ParamsARun<T, I>(a.tabA, J, f).set_p(x, c, (T)pxc.re, (T)pxc.im);
    if (a.pinvH) {  // (P^{-H})_{xc} = conj(C_xc / det P)
      cpx<double> cxc = C[0][0];
#pragma unroll
      for (int r = 0; r < I; ++r)
#pragma unroll
        for (int s = 0; s < I; ++s)
          if (r == x && s == c) cxc = C[r][s];
      const double inv = 1.0 / d2;
      const cpx<double> q = cconj(cmul(cxc, mk(det.re * inv, -det.im * inv)));
      reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I2 + lane] = make_double2(q.re, q.im);
    }
  }
  if (lane == 0) {
    if (bad) raise_status(a.status, kDevNonfinite, f);
    if (singular) raise_status(a.status, kDevSingular, f);
    atomicAdd(a.ops, p_update_inversions(a, I));
    a.logdet[f] = log(d2);
  }
}

// Newton's method for I > 4: the 2 I^2 = 128 real unknowns do not fit one
// warp, so one CTA per problem holds the system in shared memory and thread
// l < 2 I^2 owns column l (thread 2 I^2 the right-hand side): each builds its
// column of H (the closed form above), the CTA projects it off the phase
// turns as the I <= 4 kernel does, and solves by Gauss-Jordan with partial
// pivoting, every thread eliminating in its own column against a copy of
// the pivot column.  P^{-1} and the final P^{-H} and ln|det P|^2 come from
// warp 0 (pinvh_from_columns).
template <int I>
struct NewtonBig {
  static constexpr int I2 = I * I, n = 2 * I2, LD = n + 1;
  static constexpr int THREADS = n + 32;  // columns 0 .. n (the right-hand side); the rest idle in the solve
  // shared memory, in doubles: the system [n][LD] (column n: right-hand side),
  // the pivot column, V_i / N packed, P, Q = P^{-1}, G (complex I x I), W = H U
  // [n][I], S [I][I], U^T g, the column norms, the gradient [n]
  static constexpr int OFF_COLK = n * LD;
  static constexpr int OFF_V = OFF_COLK + n;
  static constexpr int OFF_PQG = (OFF_V + I * I2 + 1) / 2 * 2;  // 16-byte aligned
  static constexpr int OFF_W = OFF_PQG + 3 * 2 * I2;
  static constexpr int OFF_S = OFF_W + n * I;
  static constexpr int OFF_UG = OFF_S + I * I;
  static constexpr int OFF_NRM = OFF_UG + I;
  static constexpr int OFF_GR = OFF_NRM + I;
  static constexpr int OFF_M = (OFF_GR + n + 1) / 2 * 2;  // pinvh_from_columns' buffers
  static constexpr int BYTES = OFF_M * (int)sizeof(double) + BigLane<I>::SMEM;
};

template <typename T, int I>
__global__ void __launch_bounds__(NewtonBig<I>::THREADS) k_psolve_newton_big(FastArgs a) {
  using NB = NewtonBig<I>;
  constexpr int I2 = NB::I2, n = NB::n, LD = NB::LD, NV = I * I2, NT = NB::THREADS;
  extern __shared__ __align__(16) unsigned char nsm[];
  double* M = reinterpret_cast<double*>(nsm);
  double* colk = M + NB::OFF_COLK;
  double* sV = M + NB::OFF_V;
  cpx<double>* sP = reinterpret_cast<cpx<double>*>(M + NB::OFF_PQG);  // [x][c]
  cpx<double>* sQ = sP + I2;
  cpx<double>* sG = sQ + I2;
  double* W = M + NB::OFF_W;
  double* S = M + NB::OFF_S;
  double* Ug = M + NB::OFF_UG;
  double* nrm = M + NB::OFF_NRM;
  double* gr = M + NB::OFF_GR;
  cpx<double>* Mb = reinterpret_cast<cpx<double>*>(M + NB::OFF_M);
  __shared__ int s_piv, s_bad, s_sing;
  if (a.trace && blockIdx.x == gridDim.x - 1) {  // the trace block (one warp's work)
    if (threadIdx.x < 32) finalize_trace(a);
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int f = blockIdx.x;
  const Partition pt = a.part;
  const int J = a.J;
  if (tid == 0) {
    s_bad = 0;
    s_sing = 0;
  }
  __syncthreads();
  if (a.lam_next) {  // commit the new Lambda (computed during pass B)
    ParamsARun<T, I> ta(a.tabA, J, f);
    for (int q = tid; q < J * I; q += NT) {
      const double l = __ldcg(a.lam_next + (size_t)f * J * I + q);
      a.lam[(size_t)f * J * I + q] = l;
      ta.set_lam(q / I, q % I, (T)l);
    }
  }
  {
    const int ns = pt.nslots(f);
    const double* base = a.part_buf + ((size_t)f * pt.max_slots) * NV;
    for (int q = tid; q < NV; q += NT) {
      double sum = 0.0;
      for (int k = 0; k < ns; ++k) sum += __ldcg(base + (size_t)k * NV + q);
      sum *= pt.inv_n(f);
      if (!isfinite(sum)) s_bad = 1;
      sV[q] = sum;
    }
  }
  if (tid < I2) {
    const double2 q = __ldcg(reinterpret_cast<const double2*>(a.P) + (size_t)f * I2 + tid);
    sP[tid] = mk(q.x, q.y);
  }
  __syncthreads();
  auto Vget = [&](int c, int r, int s2) -> cpx<double> {  // [V_c]_{r s2}
    const double* v = sV + c * I2;
    if (r == s2) return mk(v[r], 0.0);
    const int lo = r < s2 ? r : s2, hi = r < s2 ? s2 : r;
    const int m = I + 2 * (lo * (2 * I - lo - 1) / 2 + (hi - lo - 1));
    return r < s2 ? mk(v[m], v[m + 1]) : mk(v[m], -v[m + 1]);
  };
  // u_i at coordinate k (nonzero where c_k = i): the direction i p_i, normalised
  auto U = [&](int i, int k) -> double {
    const int ak = (k % I2) / I, ck = k % I;
    if (ck != i) return 0.0;
    const cpx<double> pv = sP[ak * I + i];
    return (k >= I2 ? pv.re : -pv.im) * nrm[i];
  };
  const int l = tid;  // the column this thread owns (l == n: the right-hand side)
  const int al = (l % I2) / I, cl = l % I;
  const bool iml = l >= I2;
  const int g8 = lane / I, i8 = lane % I;  // warp 0's lane (group, column) for the inverses
  cpx<double>* Mg = Mb + (size_t)(g8 < BigLane<I>::G ? g8 : BigLane<I>::G) * I * BigLane<I>::LDM;

  for (int step = 0; step < a.K; ++step) {
    if (warp == 0) {  // Q = P^{-1} = (P^{-H})^H from the columns of P
      cpx<double> x[I];
#pragma unroll
      for (int r = 0; r < I; ++r) x[r] = sP[r * I + i8];
      bool sing = false;
      pinvh_from_columns<I>(x, Mg, g8, i8, sing);
      if (g8 == 0) {
#pragma unroll
        for (int r = 0; r < I; ++r) sQ[i8 * I + r] = cconj(x[r]);  // Q_{i r} = conj((P^{-H})_{r i})
        if (sing) s_sing = 1;
      }
    }
    __syncthreads();
    if (tid < I2) {  // G_xc = conj(Q_cx) - sum_b [V_c]_{xb} P_bc
      const int x = tid / I, c = tid % I;
      cpx<double> sum = cconj(sQ[c * I + x]);
      for (int b = 0; b < I; ++b) sum = csub(sum, cmul(Vget(c, x, b), sP[b * I + c]));
      sG[x * I + c] = sum;
    } else if (tid < I2 + I) {
      const int i = tid - I2;
      double s2 = 0.0;
      for (int r = 0; r < I; ++r) s2 += cabs2(sP[r * I + i]);
      nrm[i] = 1.0 / sqrt(s2);
    }
    __syncthreads();
    // column l of H and the gradient at l
    if (l < n) {
      cpx<double> ql[I], qr[I], vl[I];
#pragma unroll
      for (int x = 0; x < I; ++x) {
        ql[x] = sQ[cl * I + x];  // Q_{c_l, x}
        qr[x] = sQ[x * I + al];  // Q_{x, a_l}
        vl[x] = Vget(cl, x, al);
      }
      const cpx<double> phl = iml ? mk(0.0, 1.0) : mk(1.0, 0.0);
      for (int k = 0; k < n; ++k) {
        const int ak = (k % I2) / I, ck = k % I;
        const cpx<double> phk = k >= I2 ? mk(0.0, 1.0) : mk(1.0, 0.0);
        cpx<double> qa = ql[0], qb = qr[0], va = vl[0];
#pragma unroll
        for (int x = 1; x < I; ++x) {
          if (x == ak) {
            qa = ql[x];
            va = vl[x];
          }
          if (x == ck) qb = qr[x];
        }
        double h = -2.0 * cmul(cmul(phk, phl), cmul(qa, qb)).re;
        if (ck == cl) h -= 2.0 * cmul(cmul(cconj(phk), phl), va).re;
        M[k * LD + l] = h;
      }
      const cpx<double> gk = sG[al * I + cl];
      gr[l] = 2.0 * (iml ? gk.im : gk.re);
    }
    __syncthreads();
    // W = H U (row l from column l, H symmetric): u_i is supported on c_k = i
    if (l < n) {
      for (int i = 0; i < I; ++i) {
        double sum = 0.0;
        for (int half = 0; half < 2; ++half)
          for (int x = 0; x < I; ++x) {
            const int k = half * I2 + x * I + i;
            sum = fma(M[k * LD + l], U(i, k), sum);
          }
        W[l * I + i] = sum;
      }
    }
    __syncthreads();
    if (tid < I * I) {  // S = U^T W
      const int i = tid / I, j = tid % I;
      double sum = 0.0;
      for (int half = 0; half < 2; ++half)
        for (int x = 0; x < I; ++x) {
          const int k = half * I2 + x * I + i;
          sum = fma(U(i, k), W[k * I + j], sum);
        }
      S[tid] = sum;
    } else if (tid < I * I + I) {  // U^T g
      const int i = tid - I * I;
      double sum = 0.0;
      for (int half = 0; half < 2; ++half)
        for (int x = 0; x < I; ++x) {
          const int k = half * I2 + x * I + i;
          sum = fma(U(i, k), gr[k], sum);
        }
      Ug[i] = sum;
    }
    __syncthreads();
    // column l of Q' H Q' - Pi = H e_l - U w_l - W u_l + U (S u_l - u_l); the right-hand side -Q' g
    if (l < n) {
      double ul[I], wl[I], su[I];
#pragma unroll
      for (int i = 0; i < I; ++i) {
        ul[i] = U(i, l);
        wl[i] = W[l * I + i];
      }
#pragma unroll
      for (int i = 0; i < I; ++i) {
        double t = -ul[i];
#pragma unroll
        for (int j = 0; j < I; ++j) t = fma(S[i * I + j], ul[j], t);
        su[i] = t;
      }
      for (int k = 0; k < n; ++k) {
        double t = M[k * LD + l];
#pragma unroll
        for (int j = 0; j < I; ++j) {
          const double ujk = U(j, k);
          t = fma(-W[k * I + j], ul[j], t);
          t = fma(-ujk, wl[j], t);
          t = fma(ujk, su[j], t);
        }
        M[k * LD + l] = t;
      }
    } else if (l == n) {
      for (int k = 0; k < n; ++k) {
        double r = gr[k];
#pragma unroll
        for (int j = 0; j < I; ++j) r = fma(-U(j, k), Ug[j], r);
        M[k * LD + n] = -r;
      }
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting on [M | right-hand side]
    for (int k = 0; k < n; ++k) {
      if (warp == 0) {
        double best = -1.0;
        int p = k;
        for (int r = k + lane; r < n; r += 32) {
          const double m = fabs(M[r * LD + k]);
          if (m > best) {
            best = m;
            p = r;
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {  // the largest, the smallest row among equals
          const double ob = __shfl_xor_sync(0xffffffffu, best, off);
          const int op = __shfl_xor_sync(0xffffffffu, p, off);
          if (ob > best || (ob == best && op < p)) {
            best = ob;
            p = op;
          }
        }
        if (lane == 0) s_piv = p;
      }
      __syncthreads();
      const int p = s_piv;
      if (l <= n && p != k) {
        const double t = M[k * LD + l];
        M[k * LD + l] = M[p * LD + l];
        M[p * LD + l] = t;
      }
      __syncthreads();
      if (tid < n) colk[tid] = M[tid * LD + k];
      __syncthreads();
      const double piv = colk[k];
      if (tid == 0 && (!(piv != 0.0) || !isfinite(piv))) s_sing = 1;
      if (l <= n) {
        const double t = M[k * LD + l] / piv;
        for (int r = 0; r < n; ++r)
          if (r != k) M[r * LD + l] = fma(-colk[r], t, M[r * LD + l]);
        M[k * LD + l] = t;
      }
      __syncthreads();
    }
    // P += mu sum_k s_k E_k (s = the right-hand side column)
    if (tid < I2) {
      const double sr = M[tid * LD + n], si = M[(I2 + tid) * LD + n];
      sP[tid] = mk(sP[tid].re + a.mu * sr, sP[tid].im + a.mu * si);
    }
    __syncthreads();
  }

  // the new P (and the pass-A table), its P^{-H} and ln|det P|^2
  if (warp == 0) {
    cpx<double> x[I];
#pragma unroll
    for (int r = 0; r < I; ++r) x[r] = sP[r * I + i8];
    if (g8 == 0) {
      ParamsARun<T, I> ta(a.tabA, J, f);
#pragma unroll
      for (int r = 0; r < I; ++r) {
        reinterpret_cast<double2*>(a.P)[(size_t)f * I2 + r * I + i8] = make_double2(x[r].re, x[r].im);
        ta.set_p(r, i8, (T)x[r].re, (T)x[r].im);
      }
    }
    bool sing = false;
    const double det2 = pinvh_from_columns<I>(x, Mg, g8, i8, sing);
    if (g8 == 0) {
      if (a.pinvH) {
#pragma unroll
        for (int r = 0; r < I; ++r)
          reinterpret_cast<double2*>(a.pinvH)[(size_t)f * I2 + r * I + i8] = make_double2(x[r].re, x[r].im);
      }
      if (sing) s_sing = 1;
    }
    __syncwarp();
    if (lane == 0) {
      if (s_bad) raise_status(a.status, kDevNonfinite, f);
      if (s_sing || !(det2 > 0.0)) raise_status(a.status, kDevSingular, f);
      atomicAdd(a.ops, p_update_inversions(a, I));
      a.logdet[f] = log(det2);
    }
  }
}

}  // namespace ffca
