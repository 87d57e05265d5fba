// Adjoint kernels: gradients of two losses of the model parameters
// Psi = (v, Lambda, P) at fixed data, with the posteriors recomputed per
// time-frequency point (nothing is stored from the iterations).
//
//   NLL = -L2 (Eq. L2), per point I ln(pi) - ln|det P|^2
//         + sum_i (ln sigma_i + |y~_i|^2 / sigma_i), y~ = P^H y,
//         sigma_i = sum_j v_j lambda_ji:
//     t_i = 1/sigma_i - |y~_i|^2 / sigma_i^2
//     dNLL/dv_j = sum_i lambda_ji t_i,  dNLL/dlambda_ji = sum_n v_j t_i,
//     dNLL/dP^* = -N P^{-H} + sum_n y y^H P diag(1/sigma)   (minus Eq. partialP)
//   SE = sum_{j,n} |x^_j - s_j|^2 with the Wiener estimate x^_j =
//        Q (g_j * y~), Q = P^{-H}, g_ji = v_j lambda_ji / sigma_i (Eq. MMSE0
//        with Eq. covmodelprop), s_j the reference source images:
//     e_j = x^_j - s_j, b_j = Q^H e_j, G_ji = 2 Re(conj(b_ji) y~_i),
//     h_i = sum_j G_ji g_ji, w_ji = (G_ji - h_i) / sigma_i
//     dSE/dv_j = sum_i lambda_ji w_ji,  dSE/dlambda_ji = sum_n v_j w_ji,
//     dSE/dP^* = sum_n sum_j (y (g_j * b_j)^H - x^_j b_j^H)
// dP is the conjugate Wirtinger derivative: dLoss = 2 Re sum conj(dP) dP.
//
// k_adj streams y, v (and s) once: one CTA per contiguous unit range of pass
// A's partition (uniform for one mixture, ragged for a batch), 256 threads, per-thread sums over the range's frames of
// each frequency, a block reduction per frequency segment into that
// frequency's slot (deterministic, no atomics).  k_adj_final sums the slots
// per frequency (FP64, slot order) and adds the closed-form terms.
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

// Problems p = (mixture, frequency) of pass A's partition: uniform for one
// mixture, ragged for a batch (mixture-major blocks, as the estimation).
struct AdjArgs {
  Partition part;        // pass A's: F problems (frames, rows and offsets per problem)
  int F, N, ld;
  const void* y;         // per mixture [I][Fm][ld_m] complex
  const void* v;         // per mixture [J][Fm][ld_m] real
  const double* lam;     // [F][J][I]
  const double* P;       // [F][I][I] complex
  const double* pinvH;   // [F][I][I] complex, P^{-H} (k_prep)
  const double* logdet;  // [F] ln|det P|^2 (k_prep)
  const void* s;         // SE: per mixture [J][I][Fm][ld_m] complex reference source images
  void* dv;              // as v: frames < N_m written (and the rest of their vector units as 0)
  double* dlam;          // [F][J][I]
  double* dP;            // [F][I][I] complex
  double* part_buf;      // [F][max_slots][NV]
  double* lossf;         // [F] per-problem loss
  double* loss;          // [1] total
  unsigned* gcnt;        // arrival counter of k_adj_final
  unsigned* status;
};

template <int I, int J, bool SE>
struct AdjShape {
  static constexpr int NA = J * I;          // dlambda
  static constexpr int NP = 2 * I * I;      // dP^* (re, im), [a][i] row-major
  static constexpr int NL = SE ? 1 : 2;     // SE | NLL: sum |y~|^2/sigma, sum log2 sigma
  static constexpr int NV = NA + NP + NL;
};

template <typename T, int I, int J, bool SE>
__global__ void __launch_bounds__(kBlock) k_adj(AdjArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  constexpr int FU = Vec<T>::FU;
  using S = AdjShape<I, J, SE>;
  constexpr int NA = S::NA, NV = S::NV;
  using Red = ButterflyReduce<T, NV, kWarps, false>;
  __shared__ typename Red::Smem red;
  __shared__ double sP[I][I][2], sQ[I][I][2];
  __shared__ double sLam[J][I];

  const Partition pt = a.part;
  const long long u0 = pt.block_start(blockIdx.x), u1 = pt.block_start(blockIdx.x + 1);
  const long long row = a.ld / FU;
  const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y);
  const VV* __restrict__ v = reinterpret_cast<const VV*>(a.v);
  const VY* __restrict__ s = reinterpret_cast<const VY*>(a.s);
  VV* __restrict__ dv = reinterpret_cast<VV*>(a.dv);

  for (long long u = u0; u < u1;) {
    // problem f (a frequency of one mixture) and its rows: mixture-major
    // blocks at frame offset `off`, rows of rlen units (the single-mixture
    // case: off = 0, rlen = ld / FU, Fm = F)
    const int f = pt.problem_of(u);
    const long long us = pt.start(f);
    const int k0 = (int)(u - us);
    const int k1 = (int)(min(pt.start(f + 1), u1) - us);
    const int Np = pt.frames(f);
    const long long rlen = pt.row_len(f, row * FU) / FU;
    const long long off = pt.frame_off(f) / FU;
    const long long r0 = (long long)pt.freq(f) * rlen;
    const size_t rstr = (size_t)pt.Fm * rlen;  // from one mic's (source's) row to the next
    const VY* __restrict__ yf = y + (size_t)I * pt.Fm * off + r0;
    const VV* __restrict__ vf = v + (size_t)J * pt.Fm * off + r0;
    const VY* __restrict__ sf = SE ? s + (size_t)J * I * pt.Fm * off + r0 : nullptr;
    VV* __restrict__ dvf = dv + (size_t)J * pt.Fm * off + r0;
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
    T lam[J][I];
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int i = 0; i < I; ++i) lam[j][i] = (T)sLam[j][i];
    auto Pc = [&](int r, int c) { return mk<T>((T)sP[r][c][0], (T)sP[r][c][1]); };
    auto Qc = [&](int r, int c) { return mk<T>((T)sQ[r][c][0], (T)sQ[r][c][1]); };

    T acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = (T)0;

    for (int k = k0 + threadIdx.x; k < k1; k += kBlock) {
      VY yu[I];
      VV vu[J], dvu[J];
#pragma unroll
      for (int m = 0; m < I; ++m) yu[m] = yf[m * rstr + k];
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = vf[j * rstr + k];
#pragma unroll
      for (int e = 0; e < FU; ++e) {
        const bool valid = k * FU + e < Np;
        cpx<T> ym[I], yt[I];
#pragma unroll
        for (int m = 0; m < I; ++m) ym[m] = valid ? yframe(yu[m], e) : mk<T>(0, 0);
#pragma unroll
        for (int i = 0; i < I; ++i) {
          cpx<T> t = mk<T>(0, 0);
#pragma unroll
          for (int m = 0; m < I; ++m) cfmac(t, Pc(m, i), ym[m]);  // y~_i = sum_m conj(P_mi) y_m
          yt[i] = t;
        }
        T vj[J], sg[I], r[I];
#pragma unroll
        for (int j = 0; j < J; ++j) vj[j] = valid ? vframe(vu[j], e) : (T)1;
#pragma unroll
        for (int i = 0; i < I; ++i) {
          T t = vj[0] * lam[0][i];
#pragma unroll
          for (int j = 1; j < J; ++j) t = fma(vj[j], lam[j][i], t);
          sg[i] = t;
          r[i] = recip(t);
        }
        const T z = valid ? (T)1 : (T)0;  // padding frames contribute nothing
        if constexpr (!SE) {
          T t[I];
#pragma unroll
          for (int i = 0; i < I; ++i) {
            const T e2 = cabs2(yt[i]);
            t[i] = z * r[i] * fma(-e2, r[i], (T)1);
            acc[NV - 2] = fma(e2, r[i] * z, acc[NV - 2]);
            acc[NV - 1] += z * (sizeof(T) == 4 ? (T)__log2f((float)sg[i]) : (T)log2((double)sg[i]));
          }
#pragma unroll
          for (int j = 0; j < J; ++j) {
            T d = (T)0;
#pragma unroll
            for (int i = 0; i < I; ++i) {
              d = fma(lam[j][i], t[i], d);
              acc[j * I + i] = fma(vj[j], t[i], acc[j * I + i]);
            }
            vset(dvu[j], e, d);
          }
          // column i of sum_n y y^H P diag(1/sigma): y conj(y~_i) / sigma_i
#pragma unroll
          for (int m = 0; m < I; ++m)
#pragma unroll
            for (int i = 0; i < I; ++i) {
              const cpx<T> c = cmulc(yt[i], ym[m]);  // conj(y~_i) y_m
              acc[NA + 2 * (m * I + i)] = fma(c.re, r[i], acc[NA + 2 * (m * I + i)]);
              acc[NA + 2 * (m * I + i) + 1] = fma(c.im, r[i], acc[NA + 2 * (m * I + i) + 1]);
            }
        } else {
          T g[J][I], G[J][I];
          cpx<T> xh[J][I], b[J][I];
          T se = (T)0;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            VY su[I];
#pragma unroll
            for (int m = 0; m < I; ++m) su[m] = sf[(size_t)(j * I + m) * rstr + k];
#pragma unroll
            for (int i = 0; i < I; ++i) g[j][i] = vj[j] * lam[j][i] * r[i];
            cpx<T> err[I];
#pragma unroll
            for (int rr = 0; rr < I; ++rr) {  // x^_j = Q (g_j * y~)
              cpx<T> x = mk<T>(0, 0);
#pragma unroll
              for (int i = 0; i < I; ++i) cfma(x, Qc(rr, i), cscale(yt[i], g[j][i]));
              xh[j][rr] = x;
              const cpx<T> sv = valid ? yframe(su[rr], e) : mk<T>(0, 0);
              err[rr] = csub(x, sv);
              se = fma(z, cabs2(err[rr]), se);
            }
#pragma unroll
            for (int i = 0; i < I; ++i) {  // b_j = Q^H e_j
              cpx<T> t = mk<T>(0, 0);
#pragma unroll
              for (int rr = 0; rr < I; ++rr) cfmac(t, Qc(rr, i), err[rr]);
              b[j][i] = t;
              const cpx<T> cb = cmulc(t, yt[i]);  // conj(b_ji) y~_i
              G[j][i] = (T)2 * cb.re;
            }
          }
          acc[NV - 1] += se;
          T h[I];
#pragma unroll
          for (int i = 0; i < I; ++i) {
            T t = (T)0;
#pragma unroll
            for (int j = 0; j < J; ++j) t = fma(G[j][i], g[j][i], t);
            h[i] = t;
          }
#pragma unroll
          for (int j = 0; j < J; ++j) {
            T d = (T)0;
#pragma unroll
            for (int i = 0; i < I; ++i) {
              const T w = z * (G[j][i] - h[i]) * r[i];
              d = fma(lam[j][i], w, d);
              acc[j * I + i] = fma(vj[j], w, acc[j * I + i]);
            }
            vset(dvu[j], e, d);
          }
          // sum_j (y (g_j * b_j)^H - x^_j b_j^H): entry [a][c]
#pragma unroll
          for (int m = 0; m < I; ++m)
#pragma unroll
            for (int c = 0; c < I; ++c) {
              cpx<T> t = mk<T>(0, 0);
#pragma unroll
              for (int j = 0; j < J; ++j) {
                const cpx<T> bc = cconj(b[j][c]);
                t = cadd(t, cmul(ym[m], cscale(bc, g[j][c])));
                t = csub(t, cmul(xh[j][m], bc));
              }
              acc[NA + 2 * (m * I + c)] = fma(z, t.re, acc[NA + 2 * (m * I + c)]);
              acc[NA + 2 * (m * I + c) + 1] = fma(z, t.im, acc[NA + 2 * (m * I + c) + 1]);
            }
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j) dvf[j * rstr + k] = dvu[j];
    }
    // the segment's sums into slot (f, this CTA)
    const int slot = (int)blockIdx.x - pt.first_block(f);
    double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * NV;
    T lo[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) lo[q] = (T)0;
    Red::run(acc, lo, red, out);
    u += k1 - k0;
  }
}

// The adjoint for I > 4: the per-point state (I^2 + J I sums of dP^* and
// dLambda, the Wiener estimates of J sources) does not fit one thread, so
// each unit is shared by I threads as in pass B's I > 4 form.  Thread e owns
// index i = e: y~_e, sigma_e, r_e, the Lambda sums of column e, column e of
// dP^* (I complex sums), and the loss parts of i = e.  Sums over i (dv_j;
// the Wiener estimates x^_j = Q (g_j * y~) and b_j = Q^H e_j of the squared
// error) go through the unit's lanes by shuffles: thread e forms row e of
// x^_j from the gathered g_ji y~_i, and its entry b_je from the gathered
// rows of e_j.  The slot layout is k_adj's: dlambda, dP^* (re, im) [a][i],
// then the loss parts.
template <int I, int J, bool SE>
struct AdjBig {
  using S = AdjShape<I, J, SE>;
  static constexpr int NVT = J + 2 * I + S::NL;  // values per thread
  // slot index of thread e's value v, or -1 (the loss parts of threads
  // e > 0, which the reduction leaves in thread 0)
  __device__ static int out_index(int e, int v) {
    if (v < J) return v * I + e;
    if (v < J + 2 * I) {
      const int m = (v - J) / 2, comp = (v - J) % 2;
      return S::NA + 2 * (m * I + e) + comp;
    }
    return e == 0 ? S::NA + S::NP + (v - J - 2 * I) : -1;
  }
};

template <typename T>
__device__ inline cpx<T> shfl_cx(cpx<T> z, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, z.re, src), __shfl_sync(0xffffffffu, z.im, src));
}

template <typename T, int I, int J, bool SE>
__global__ void __launch_bounds__(kBlock) k_adj_big(AdjArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  constexpr int FU = Vec<T>::FU;
  using S = AdjShape<I, J, SE>;
  using AB = AdjBig<I, J, SE>;
  constexpr int NVT = AB::NVT;
  constexpr int UG = kBlock / I;  // units in flight per CTA
  static_assert(kBlock % I == 0 && 32 % I == 0 && J <= I, "I must divide the block and the warp");
  __shared__ T red[kWarps][I * NVT];
  __shared__ double sP[I][I][2], sQ[I][I][2];
  __shared__ double sLam[J][I];

  const Partition pt = a.part;
  const long long u0 = pt.block_start(blockIdx.x), u1 = pt.block_start(blockIdx.x + 1);
  const long long row = a.ld / FU;
  const VY* __restrict__ y = reinterpret_cast<const VY*>(a.y);
  const VV* __restrict__ v = reinterpret_cast<const VV*>(a.v);
  const VY* __restrict__ s = reinterpret_cast<const VY*>(a.s);
  VV* __restrict__ dv = reinterpret_cast<VV*>(a.dv);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = threadIdx.x % I, ul = threadIdx.x / I;
  const int gl = lane & ~(I - 1);  // first lane of this unit's I threads

  for (long long u = u0; u < u1;) {
    const int f = pt.problem_of(u);
    const long long us = pt.start(f);
    const int k0 = (int)(u - us);
    const int k1 = (int)(min(pt.start(f + 1), u1) - us);
    const int Np = pt.frames(f);
    const long long rlen = pt.row_len(f, row * FU) / FU;
    const long long off = pt.frame_off(f) / FU;
    const long long r0 = (long long)pt.freq(f) * rlen;
    const size_t rstr = (size_t)pt.Fm * rlen;
    const VY* __restrict__ yf = y + (size_t)I * pt.Fm * off + r0;
    const VV* __restrict__ vf = v + (size_t)J * pt.Fm * off + r0;
    const VY* __restrict__ sf = SE ? s + (size_t)J * I * pt.Fm * off + r0 : nullptr;
    VV* __restrict__ dvf = dv + (size_t)J * pt.Fm * off + r0;
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
    cpx<T> pcol[I];  // column e of P
    T lam_e[J];      // lambda_je
#pragma unroll
    for (int m = 0; m < I; ++m) pcol[m] = mk<T>((T)sP[m][e][0], (T)sP[m][e][1]);
#pragma unroll
    for (int j = 0; j < J; ++j) lam_e[j] = (T)sLam[j][e];
    auto Qc = [&](int r, int c) { return mk<T>((T)sQ[r][c][0], (T)sQ[r][c][1]); };

    T acc[NVT];
#pragma unroll
    for (int q = 0; q < NVT; ++q) acc[q] = (T)0;

    // every lane takes the same trips (the shuffles need the whole warp)
    for (int kb = k0; kb < k1; kb += UG) {
      const int k = kb + ul;
      const bool unit_ok = k < k1;
      VY yu[I];
      VV vu[J], dvu;
#pragma unroll
      for (int m = 0; m < I; ++m) yu[m] = unit_ok ? yf[m * rstr + k] : VY{};
#pragma unroll
      for (int j = 0; j < J; ++j) vu[j] = unit_ok ? vf[j * rstr + k] : VV{};
      dvu = VV{};
#pragma unroll
      for (int fr = 0; fr < FU; ++fr) {
        const bool valid = unit_ok && k * FU + fr < Np;
        const T z = valid ? (T)1 : (T)0;  // padding frames contribute nothing
        cpx<T> ym[I];
#pragma unroll
        for (int m = 0; m < I; ++m) ym[m] = valid ? yframe(yu[m], fr) : mk<T>(0, 0);
        cpx<T> yte = mk<T>(0, 0);  // y~_e = sum_m conj(P_me) y_m
#pragma unroll
        for (int m = 0; m < I; ++m) cfmac(yte, pcol[m], ym[m]);
        T vj[J];
#pragma unroll
        for (int j = 0; j < J; ++j) vj[j] = valid ? vframe(vu[j], fr) : (T)1;
        T sg = vj[0] * lam_e[0];
#pragma unroll
        for (int j = 1; j < J; ++j) sg = fma(vj[j], lam_e[j], sg);
        const T re = recip(sg);
        T dvo[J];  // this thread's term of dv_j (summed over the unit's threads below)
        if constexpr (!SE) {
          const T e2 = cabs2(yte);
          const T te = z * re * fma(-e2, re, (T)1);
          acc[J + 2 * I] = fma(e2, re * z, acc[J + 2 * I]);
          acc[J + 2 * I + 1] += z * (sizeof(T) == 4 ? (T)__log2f((float)sg) : (T)log2((double)sg));
#pragma unroll
          for (int j = 0; j < J; ++j) {
            dvo[j] = lam_e[j] * te;
            acc[j] = fma(vj[j], te, acc[j]);
          }
          // column e of sum_n y y^H P diag(1/sigma): y_m conj(y~_e) / sigma_e
#pragma unroll
          for (int m = 0; m < I; ++m) {
            const cpx<T> c = cmulc(yte, ym[m]);  // conj(y~_e) y_m
            acc[J + 2 * m] = fma(c.re, re, acc[J + 2 * m]);
            acc[J + 2 * m + 1] = fma(c.im, re, acc[J + 2 * m + 1]);
          }
        } else {
          // row e of x^_j = Q (g_j * y~), g_ji = v_j lambda_ji r_i, from the gathered y~_i and r_i
          cpx<T> xh[J];
#pragma unroll
          for (int j = 0; j < J; ++j) xh[j] = mk<T>(0, 0);
#pragma unroll
          for (int i = 0; i < I; ++i) {
            const cpx<T> yti = shfl_cx(yte, gl | i);
            const T ri = __shfl_sync(0xffffffffu, re, gl | i);
            const cpx<T> q = Qc(e, i);
#pragma unroll
            for (int j = 0; j < J; ++j) cfma(xh[j], q, cscale(yti, vj[j] * (T)sLam[j][i] * ri));
          }
          // e_je = x^_je - s_je; b_je = sum_m conj(Q_me) e_jm from the gathered rows
          cpx<T> err[J], b[J];
          T se = (T)0;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const cpx<T> sv = valid ? yframe(sf[(size_t)(j * I + e) * rstr + k], fr) : mk<T>(0, 0);
            err[j] = csub(xh[j], sv);
            se = fma(z, cabs2(err[j]), se);
            b[j] = mk<T>(0, 0);
          }
          acc[J + 2 * I] += se;
#pragma unroll
          for (int m = 0; m < I; ++m) {
            const cpx<T> q = Qc(m, e);
#pragma unroll
            for (int j = 0; j < J; ++j) cfmac(b[j], q, shfl_cx(err[j], gl | m));
          }
          T g[J], G[J], h = (T)0;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            g[j] = vj[j] * lam_e[j] * re;
            G[j] = (T)2 * cmulc(b[j], yte).re;  // 2 Re(conj(b_je) y~_e)
            h = fma(G[j], g[j], h);
          }
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const T w = z * (G[j] - h) * re;
            dvo[j] = lam_e[j] * w;
            acc[j] = fma(vj[j], w, acc[j]);
          }
          // column e of sum_j (y (g_j * b_j)^H - x^_j b_j^H): entry [a][e], x^_ja from row a's lane
#pragma unroll
          for (int aa = 0; aa < I; ++aa) {
            cpx<T> t = mk<T>(0, 0);
#pragma unroll
            for (int j = 0; j < J; ++j) {
              const cpx<T> bc = cconj(b[j]);
              t = cadd(t, cmul(ym[aa], cscale(bc, g[j])));
              t = csub(t, cmul(shfl_cx(xh[j], gl | aa), bc));
            }
            acc[J + 2 * aa] = fma(z, t.re, acc[J + 2 * aa]);
            acc[J + 2 * aa + 1] = fma(z, t.im, acc[J + 2 * aa + 1]);
          }
        }
        // dv_j = sum over the unit's threads; thread j keeps frame fr of dv_j
#pragma unroll
        for (int j = 0; j < J; ++j) {
          T d = dvo[j];
#pragma unroll
          for (int off = 1; off < I; off <<= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
          if (j == e) vset(dvu, fr, d);
        }
      }
      if (unit_ok && e < J) dvf[e * rstr + k] = dvu;
    }
    // the segment's sums into slot (f, this CTA): the loss parts over the
    // unit's threads, the lanes with the same e, then the warps (FP64)
#pragma unroll
    for (int q = J + 2 * I; q < NVT; ++q)
#pragma unroll
      for (int off = 1; off < I; off <<= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
#pragma unroll
    for (int off = I; off < 32; off <<= 1)
#pragma unroll
      for (int q = 0; q < NVT; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (lane < I) {
#pragma unroll
      for (int q = 0; q < NVT; ++q) red[warp][lane * NVT + q] = acc[q];
    }
    __syncthreads();
    const int slot = (int)blockIdx.x - pt.first_block(f);
    double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * S::NV;
    for (int x = threadIdx.x; x < I * NVT; x += kBlock) {
      const int o = AB::out_index(x / NVT, x % NVT);
      if (o < 0) continue;
      double t = 0.0;
#pragma unroll
      for (int w2 = 0; w2 < kWarps; ++w2) t += (double)red[w2][x];
      out[o] = t;
    }
    u += k1 - k0;
  }
}

// One warp per frequency: slot sums (FP64, slot order) into dlam, dP and the
// frequency's loss; the last warp adds the losses.
template <typename T, int I, int J, bool SE>
__global__ void __launch_bounds__(128) k_adj_final(AdjArgs a) {
  using S = AdjShape<I, J, SE>;
  constexpr int NA = S::NA, NP = S::NP, NV = S::NV;
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (f >= a.F) return;  // whole warps only
  const Partition pt = a.part;
  const int ns = pt.nslots(f);
  const double* base = a.part_buf + (size_t)f * pt.max_slots * NV;
  double lossv = 0.0;
  for (int q = lane; q < NV; q += 32) {
    double t = 0.0;
    for (int k = 0; k < ns; ++k) t += __ldcg(base + (size_t)k * NV + q);
    if (q < NA) {
      a.dlam[(size_t)f * NA + q] = t;
    } else if (q < NA + NP) {
      const int idx = q - NA;  // 2 (m I + i) + part
      if constexpr (!SE) t -= (double)pt.frames(f) * a.pinvH[(size_t)f * I * I * 2 + idx];
      a.dP[(size_t)f * I * I * 2 + idx] = t;
    } else if constexpr (SE) {
      lossv += t;
    } else {
      lossv += (q == NV - 2) ? t : 0.69314718055994530942 * t;
    }
  }
  // lanes holding loss terms: NV - NL .. NV - 1
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lossv += __shfl_xor_sync(0xffffffffu, lossv, off);
  if (lane == 0) {
    double lf = lossv;
    if constexpr (!SE) lf += (double)pt.frames(f) * ((double)I * kLnPi - __ldcg(a.logdet + f));
    if (!isfinite(lf)) raise_status(a.status, kDevNonfinite, f);
    a.lossf[f] = lf;
    __threadfence();
  }
  __syncwarp();
  unsigned last = 0;
  if (lane == 0) {
    last = atomicAdd(a.gcnt, 1u) == (unsigned)a.F - 1;
    if (last) *a.gcnt = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    double sacc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) sacc[u] = 0.0;
    for (int g = lane; g < a.F; g += 256) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (g + 32 * u < a.F) sacc[u] += __ldcg(a.lossf + g + 32 * u);
    }
    double t = ((sacc[0] + sacc[1]) + (sacc[2] + sacc[3])) + ((sacc[4] + sacc[5]) + (sacc[6] + sacc[7]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) *a.loss = t;
  }
}

}  // namespace ffca
