// Conventional FCA EM (Sec. 3.3) for arrays of more than four microphones.
// The per-point state of the small kernel (J packed I x I sums per thread)
// does not fit at I = 8, so the E/M steps are rearranged with exact
// identities; every point still needs the full Hermitian inverse of R.
//
// Per point, with R = sum_j v_j S_j, z = R^{-1} y (Eq. MMSE: mu_j = v_j S_j z,
// Eq. postquadexp: Phi_j = v_j S_j - v_j S_j R^{-1} v_j S_j):
//   tr(S_j^{-1} (mu_j mu_j^H + Phi_j)) = v_j^2 z^H S_j z + v_j I - v_j^2 tr(R^{-1} S_j)
// so Eq. vupdate needs no S_j^{-1}, and the Eq. Supdate numerator is
//   sum_n (mu_j mu_j^H + Phi_j) / v_j^new = S_j A_j S_j + b_j S_j,
//   A_j = sum_n (v_j^2 / v_j^new) (z z^H - R^{-1}),  b_j = sum_n v_j / v_j^new,
// whose two products per j are done once per frequency (FP64) instead of per
// point.  Operations are counted as performed: N F inversions (of R) and 2 J F
// products per iteration.
//
//   k_fca_em_big     phase 1, one thread per frame of a chunk: R, its
//                    Cholesky factor, ln det R, z, y^H z and R^{-1} into shared
//                    memory; phase 2, warp j < J per source: the v update in
//                    place and the sums A_j, b_j; per segment, warp sums into
//                    the frequency's slot, and the block's L1 terms.
//   k_fca_final_big  one warp per frequency (FP64): S_j = (S_j A_j S_j + b_j S_j)/N,
//                    the table, the frequency's L1; the last warp sums the trace.
#pragma once

#include "ffca_fca.cuh"

namespace ffca {

template <typename T, int I, int J>
struct FcaBig {
  static constexpr int NH = I * I;           // packed Hermitian: I real diagonal, (re, im) above it
  static constexpr int NA = J * (NH + 1);    // A_j and b_j per source
  static constexpr int NV = NA + 1;          // + the L1 terms (ln det R + y^H R^{-1} y)
  static constexpr int CH = kBlock;          // frames per chunk (one per thread in phase 1)
  static constexpr int REC = NH + 2 * I + 1; // per frame: R^{-1} packed, z, v slot marker
  static constexpr int SMEM = CH * (REC + J) * (int)sizeof(T);
  static_assert(J <= kWarps, "one warp per source");
};

// S_j in the per-point precision (row-major complex).
template <typename T, int I, int J>
struct FcaParamsBig {
  T s[J][I][I][2];
  static constexpr int BYTES = (int)(sizeof(T) * 2 * J * I * I);
};

template <typename T, int I, int J>
__global__ void k_fca_prep_big(FcaArgs a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.F) return;
  T* tp = reinterpret_cast<T*>(static_cast<char*>(a.tab) + (size_t)f * FcaParamsBig<T, I, J>::BYTES);
  const double* sp = a.S + (size_t)f * J * I * I * 2;
  for (int q = 0; q < J * I * I * 2; ++q) tp[q] = (T)sp[q];
}

// Warp-level sum of NV per-lane values (hi, lo) into out[0 .. NV) (double-float, lane order).
template <typename T, int NV>
__device__ inline void warp_sum_out(T (&h)[NV], double* out) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < NV; ++q) {
    T s = h[q], c = (T)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T rs = __shfl_xor_sync(0xffffffffu, s, off);
      const T rc = __shfl_xor_sync(0xffffffffu, c, off);
      if constexpr (sizeof(T) == 4) df_add(s, c, rs, rc);
      else s += rs;
    }
    if (lane == 0) out[q] = (double)s + (double)c;
  }
}

template <typename T, int I, int J, bool UPDATE>
__global__ void __launch_bounds__(kBlock) k_fca_em_big(FcaArgs a) {
  using B = FcaBig<T, I, J>;
  constexpr int NH = B::NH, NV = UPDATE ? B::NV : 1, CH = B::CH, REC = B::REC;
  extern __shared__ __align__(16) unsigned char fca_smem[];
  T* rec = reinterpret_cast<T*>(fca_smem);      // [CH][REC]
  T* vrec = rec + (size_t)CH * REC;             // [CH][J] current v
  __shared__ T sS[J][I][I][2];
  __shared__ double lpart[kWarps];

  const Partition pt = a.part;
  const long long total = (long long)pt.F * pt.Uf;
  const long long u0 = (long long)blockIdx.x * pt.upb;
  const long long u1 = min(u0 + pt.upb, total);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ y = reinterpret_cast<const T*>(a.y);  // complex interleaved
  T* __restrict__ v = reinterpret_cast<T*>(a.v);

  // frames, not vector units: the partition counts units of FU frames
  constexpr int FU = Vec<T>::FU;
  for (long long u = u0; u < u1;) {
    const int f = (int)(u / pt.Uf);
    const int k0 = (int)(u - (long long)f * pt.Uf);
    const int k1 = (int)min((long long)pt.Uf, k0 + (u1 - u));
    const int n_lo = k0 * FU, n_hi = min(k1 * FU, a.N);
    __syncthreads();
    {
      const T* src = reinterpret_cast<const T*>(static_cast<const char*>(a.tab) +
                                                 (size_t)f * FcaParamsBig<T, I, J>::BYTES);
      T* dst = &sS[0][0][0][0];
      for (int t = threadIdx.x; t < J * I * I * 2; t += kBlock) dst[t] = src[t];
    }
    __syncthreads();
    T acc[UPDATE ? NH + 1 : 1];
#pragma unroll
    for (int q = 0; q < (UPDATE ? NH + 1 : 1); ++q) acc[q] = (T)0;
    T lsum = (T)0;
    for (int c0 = n_lo; c0 < n_hi; c0 += CH) {
      // ---- phase 1: one frame per thread
      const int n = c0 + threadIdx.x;
      if (n < n_hi) {
        cpx<T> yv[I];
#pragma unroll
        for (int m = 0; m < I; ++m) {
          const size_t o = (((size_t)m * pt.F + f) * a.ld + n) * 2;
          yv[m] = mk<T>(y[o], y[o + 1]);
        }
        T vj[J];
#pragma unroll
        for (int j = 0; j < J; ++j) vj[j] = v[((size_t)j * pt.F + f) * a.ld + n];
        // R (lower triangle) and its Cholesky factor L, in place
        cpx<T> L[I][I];
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = 0; c <= r; ++c) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int j = 0; j < J; ++j) {
              s.re = fma(vj[j], sS[j][r][c][0], s.re);
              s.im = fma(vj[j], sS[j][r][c][1], s.im);
            }
            L[r][c] = s;
          }
        T logdet = (T)0;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < I; ++k) {
          T d = L[k][k].re;
#pragma unroll
          for (int c = 0; c < k; ++c) d -= cabs2(L[k][c]);
          ok &= d > (T)0;
          const T lkk = sqrt(d), rl = recip(lkk);
          logdet += logx(d);
          L[k][k] = mk<T>(lkk, 0);
#pragma unroll
          for (int r = k + 1; r < I; ++r) {
            cpx<T> s = L[r][k];
#pragma unroll
            for (int c = 0; c < k; ++c) s = csub(s, cmul(L[r][c], cconj(L[k][c])));
            L[r][k] = cscale(s, rl);
          }
        }
        if (!ok) raise_status(a.status, kDevSingular, f);
        // W = L^{-1} (lower), R^{-1} = W^H W
        cpx<T> W[I][I];
#pragma unroll
        for (int c = 0; c < I; ++c) {
#pragma unroll
          for (int r = 0; r < I; ++r) {
            if (r < c) continue;
            cpx<T> s = mk<T>(r == c ? (T)1 : (T)0, 0);
#pragma unroll
            for (int q = c; q < r; ++q) s = csub(s, cmul(L[r][q], W[q][c]));
            W[r][c] = cscale(s, recip(L[r][r].re));
          }
        }
        // z = R^{-1} y = W^H (W y)
        cpx<T> wy[I], z[I];
#pragma unroll
        for (int r = 0; r < I; ++r) {
          cpx<T> s = mk<T>(0, 0);
#pragma unroll
          for (int c = 0; c <= r; ++c) cfma(s, W[r][c], yv[c]);
          wy[r] = s;
        }
        T quad = (T)0;
#pragma unroll
        for (int r = 0; r < I; ++r) quad += cabs2(wy[r]);
#pragma unroll
        for (int c = 0; c < I; ++c) {
          cpx<T> s = mk<T>(0, 0);
#pragma unroll
          for (int r = c; r < I; ++r) cfmac(s, W[r][c], wy[r]);  // conj(W_rc) wy_r
          z[c] = s;
        }
        lsum += logdet + quad;
        if constexpr (UPDATE) {
          T* rp = rec + (size_t)threadIdx.x * REC;
          int e = I;
#pragma unroll
          for (int r = 0; r < I; ++r) {
            // (R^{-1})_rc = sum_q conj(W_qr) W_qc, q >= max(r, c)
            T d = (T)0;
#pragma unroll
            for (int q = r; q < I; ++q) d += cabs2(W[q][r]);
            rp[r] = d;
#pragma unroll
            for (int c = r + 1; c < I; ++c) {
              cpx<T> s = mk<T>(0, 0);
#pragma unroll
              for (int q = c; q < I; ++q) cfmac(s, W[q][r], W[q][c]);
              rp[e] = s.re;
              rp[e + 1] = s.im;
              e += 2;
            }
          }
#pragma unroll
          for (int r = 0; r < I; ++r) {
            rp[NH + 2 * r] = z[r].re;
            rp[NH + 2 * r + 1] = z[r].im;
          }
#pragma unroll
          for (int j = 0; j < J; ++j) vrec[(size_t)threadIdx.x * J + j] = vj[j];
        }
      }
      if constexpr (UPDATE) {
        __syncthreads();
        // ---- phase 2: warp j updates v_j and accumulates A_j, b_j
        if (warp < J) {
          const int j = warp;
          for (int p = lane; p < CH && c0 + p < n_hi; p += 32) {
            const T* rp = rec + (size_t)p * REC;
            const T vv = vrec[(size_t)p * J + j];
            cpx<T> zz[I];
#pragma unroll
            for (int r = 0; r < I; ++r) zz[r] = mk<T>(rp[NH + 2 * r], rp[NH + 2 * r + 1]);
            // z^H S_j z and tr(R^{-1} S_j) = sum_rc (R^{-1})_rc (S_j)_cr
            T zsz = (T)0, trs = (T)0;
            int e = I;
#pragma unroll
            for (int r = 0; r < I; ++r) {
              zsz += sS[j][r][r][0] * cabs2(zz[r]);
              trs += rp[r] * sS[j][r][r][0];
#pragma unroll
              for (int c = r + 1; c < I; ++c) {
                // z^H S z: 2 Re(conj(z_r) S_rc z_c); tr: 2 Re((R^{-1})_rc S_cr)
                const cpx<T> s_rc = mk<T>(sS[j][r][c][0], sS[j][r][c][1]);
                const cpx<T> t = cmul(cmulc(zz[r], s_rc), zz[c]);
                zsz += (T)2 * t.re;
                trs += (T)2 * (rp[e] * sS[j][c][r][0] - rp[e + 1] * sS[j][c][r][1]);
                e += 2;
              }
            }
            const T vn = (vv * vv * zsz + vv * (T)I - vv * vv * trs) * (T)(1.0 / I);
            v[((size_t)j * pt.F + f) * a.ld + c0 + p] = vn;
            const T rvn = recip(vn);
            const T g = vv * vv * rvn;
            // A_j += g (z z^H - R^{-1}) packed; b_j += v / v_new
            e = I;
#pragma unroll
            for (int r = 0; r < I; ++r) {
              acc[r] = fma(g, cabs2(zz[r]) - rp[r], acc[r]);
#pragma unroll
              for (int c = r + 1; c < I; ++c) {
                const cpx<T> t = cmulc(zz[c], zz[r]);  // z_r conj(z_c)
                acc[e] = fma(g, t.re - rp[e], acc[e]);
                acc[e + 1] = fma(g, t.im - rp[e + 1], acc[e + 1]);
                e += 2;
              }
            }
            acc[NH] = fma(vv, rvn, acc[NH]);
          }
        }
      }
      __syncthreads();  // the chunk's records are consumed
    }
    // ---- the segment's sums into slot (f, this CTA)
    const int slot = (int)blockIdx.x - pt.first_block(f);
    double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * NV;
    if constexpr (UPDATE) {
      if (warp < J) warp_sum_out<T, NH + 1>(acc, out + (size_t)warp * (NH + 1));
    }
    {
      double s = (double)lsum;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) lpart[warp] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += lpart[w];
        out[NV - 1] = t;
      }
    }
    if (UPDATE && threadIdx.x == 0 && n_hi > n_lo) atomicAdd(a.ops, (unsigned long long)(n_hi - n_lo));
    u += k1 - k0;
  }
}

// One warp per frequency (FP64): S_j = (S_j A_j S_j + b_j S_j) / N (the rearranged
// Eq. Supdate), the table, the frequency's L1 of the entering state; the last
// warp sums the trace.  With UPDATE false only the log-likelihood.
template <typename T, int I, int J, bool UPDATE>
__global__ void __launch_bounds__(128) k_fca_final_big(FcaArgs a) {
  using B = FcaBig<T, I, J>;
  constexpr int NH = B::NH, NV = UPDATE ? B::NV : 1;
  __shared__ cpx<double> sm[4][2][I][I];  // per warp: S_j, A_j
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int f = blockIdx.x * 4 + wl;
  const bool active = f < a.F;
  const Partition pt = a.part;
  const int fs = active ? f : 0;
  const int ns = pt.nslots(fs);
  const double* base = a.part_buf + (size_t)fs * pt.max_slots * NV;
  auto slot_sum = [&](int q) {
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += __ldcg(base + (size_t)k * NV + q);
    return s;
  };
  if (active && lane == 0) {
    const double lf = -(double)I * a.N * kLnPi - slot_sum(NV - 1);
    if (!isfinite(lf)) raise_status(a.status, kDevNonfinite, f);
    a.llf[f] = lf;
    __threadfence();
  }
  if constexpr (UPDATE) {
    T* tp = reinterpret_cast<T*>(static_cast<char*>(a.tab) + (size_t)fs * FcaParamsBig<T, I, J>::BYTES);
    for (int j = 0; j < J; ++j) {
      double* sp = a.S + ((size_t)fs * J + j) * I * I * 2;
      // S_j (current) and A_j (packed Hermitian) into shared memory
      for (int q = lane; q < I * I; q += 32) sm[wl][0][q / I][q % I] = mk(sp[2 * q], sp[2 * q + 1]);
      const int jb = j * (NH + 1);
      for (int q = lane; q < I * I; q += 32) {
        const int r = q / I, c = q % I;
        if (r == c) {
          sm[wl][1][r][r] = mk(slot_sum(jb + r), 0.0);
        } else if (r < c) {
          const int e = I + 2 * (r * I - r * (r + 1) / 2 + (c - r - 1));  // packed index of (r, c), r < c
          const cpx<double> z = mk(slot_sum(jb + e), slot_sum(jb + e + 1));
          sm[wl][1][r][c] = z;
          sm[wl][1][c][r] = cconj(z);
        }
      }
      const double bj = slot_sum(jb + NH);
      __syncwarp();
      cpx<double> res[(I * I + 31) / 32];
      int nr = 0;
      for (int q = lane; q < I * I; q += 32, ++nr) {
        const int r = q / I, c = q % I;
        cpx<double> s = cscale(sm[wl][0][r][c], bj);
        for (int k = 0; k < I; ++k) {
          cpx<double> t = mk(0.0, 0.0);
          for (int l = 0; l < I; ++l) t = cadd(t, cmul(sm[wl][1][k][l], sm[wl][0][l][c]));
          s = cadd(s, cmul(sm[wl][0][r][k], t));
        }
        res[nr] = cscale(s, 1.0 / a.N);
      }
      __syncwarp();
      nr = 0;
      for (int q = lane; q < I * I; q += 32, ++nr) {
        if (active) {
          sp[2 * q] = res[nr].re;
          sp[2 * q + 1] = res[nr].im;
          tp[(size_t)j * I * I * 2 + 2 * q] = (T)res[nr].re;
          tp[(size_t)j * I * I * 2 + 2 * q + 1] = (T)res[nr].im;
        }
        if (!isfinite(res[nr].re) || !isfinite(res[nr].im)) raise_status(a.status, kDevNonfinite, fs);
      }
      __syncwarp();
    }
    if (active && lane == 0) atomicAdd(a.mults, (unsigned long long)(2 * J));  // S_j A_j S_j per frequency
  }
  __syncwarp();
  unsigned last = 0;
  if (lane == 0) {
    last = atomicAdd(a.gcnt, 1u) == (unsigned)((gridDim.x * 4)) - 1;
    if (last) *a.gcnt = 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f2 = lane; f2 < a.F; f2 += 128) {
#pragma unroll
      for (int uu = 0; uu < 4; ++uu)
        if (f2 + 32 * uu < a.F) s[uu] += __ldcg(a.llf + f2 + 32 * uu);
    }
    double t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) a.trace[a.trace_slot] = t;
  }
}

}  // namespace ffca
