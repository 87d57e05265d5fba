// Hybrid iterations with each problem resident on chip: one CTA per problem
// keeps the problem's y and v in shared memory across up to kResChunk
// iterations of one launch (Sec. 4.4: the EM half, then the fixed point of
// Eq. FPI), so that a problem small enough to fit streams its data from HBM
// once per launch instead of twice per iteration, and an iteration costs no
// launch.  For problems of a few hundred to a few thousand frames, where the
// streaming passes are too short to fill the GPU.
//
//   k_resident  per iteration, the whole CTA: pass A (y~, sigma, the
//               posterior powers, v in place, the sums of Eq. Lambdaupdate
//               and of Eq. L2; per-point arithmetic in T, every thread's
//               sums over ceil(N / 256) frames in T, a butterfly over each
//               warp's lanes in T, the warps added in FP64), the
//               new Lambda and the problem's L2 of the entering state (FP64),
//               pass B (the outer product of each frame once, weighted into
//               every V_i; two sub-passes of two V_i in FP64 at I = 4, one
//               sub-pass per V_i at I = 8, one in all otherwise), then warp 0
//               runs the P step of k_psolve_ldl (L D L^H of V_i, the columns
//               V_i^{-1} [P^{-H}]_i, K sweeps, the inverse of the new P for
//               ln|det P|^2 and the next P^{-H}); at I = 3 in the layout of
//               k_psolve_wide, the work inside each V_i over the lanes, with
//               the same P^{-H} bits.  At the end v, Lambda, P,
//               P^{-H}, ln|det P|^2 and the pass-A table go back to global
//               memory; each iteration's L2 of the problem goes to hist.
//   k_res_trace one block per iteration: the problems' L2 summed in a fixed
//               order into the trace.
#pragma once

#include "ffca_big.cuh"
#include "ffca_psolve_wide.cuh"

namespace ffca {

constexpr int kResThreads = 256;
constexpr int kResWarps = kResThreads / 32;
constexpr int kResChunk = 32;          // iterations per launch
constexpr int kResSmemBudget = 200 * 1024;

struct ResArgs {
  FastArgs a;      // state, partition (problems), workspace pointers, status
  double* hist;    // [kResChunk][problems] per-iteration L2 of every problem
  int iters;       // iterations of this launch (<= kResChunk)
};

// Block sum of NV per-thread values in T: a butterfly reduce-scatter in
// each warp (31 exchanges per 32 values; lane l ends with value l of its
// chunk), then the warps' results added in FP64 in warp order.  Thread
// t < NV writes value t to out[t].  Called by the whole CTA.
template <typename T, int NV>
struct ResReduce {
  static constexpr int NC = (NV + 31) / 32;
  struct Smem {
    T v[kResWarps][NC * 32];
  };
  __device__ static void run(const T (&x)[NV], Smem& sm, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T h[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) h[k] = c * 32 + k < NV ? x[c * 32 + k] : (T)0;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < off; ++k) {
          const T keep = up ? h[k + off] : h[k];
          const T send = up ? h[k] : h[k + off];
          h[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      sm.v[warp][c * 32 + lane] = h[0];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NV; t += kResThreads) {
      double s = (double)sm.v[0][t];
#pragma unroll
      for (int w = 1; w < kResWarps; ++w) s += (double)sm.v[w][t];
      out[t] = s;
    }
    __syncthreads();
  }
};

template <typename T, int I, int J>
struct ResShape {
  static constexpr int NVA = J * I + 2;  // Lambda sums, then the quadratic and log2 parts of L2
  static constexpr int NVB = I * I;      // V_i of one i (packed Hermitian)
  // V_i summed together in one sub-pass of pass B, to keep the accumulators
  // in registers: all I for I <= 4 (FP64 I = 4: two sub-passes of two), one
  // at a time for I = 8 (64 sums each)
  static constexpr int IB = I > 4 ? 1 : ((sizeof(T) == 8 && I == 4) ? 2 : I);
  // bytes of shared memory per frame
  static constexpr int BYTES_PER_FRAME = I * (int)sizeof(cpx<T>) + J * (int)sizeof(T);
  static constexpr int max_frames() { return (kResSmemBudget / BYTES_PER_FRAME) / 4 * 4; }
};

template <typename T, int I, int J>
__global__ void __launch_bounds__(kResThreads) k_resident(ResArgs ra) {
  using RS = ResShape<T, I, J>;
  using C = cpx<T>;
  constexpr int NVA = RS::NVA, NVB = RS::NVB, NA = J * I, IB = RS::IB;
  extern __shared__ __align__(16) unsigned char res_smem[];
  __shared__ typename ResReduce<T, NVA>::Smem redA;
  __shared__ typename ResReduce<T, IB * NVB>::Smem redB;
  __shared__ double sumsA[NVA], sumsB[IB * NVB];
  __shared__ double sV[I][NVB];          // V_i / N, packed Hermitian per i
  __shared__ double sLam[J][I];          // current Lambda (FP64)
  __shared__ T sLamT[J][I];              // and in T
  __shared__ C sPT[I][I];                // P in T (per point)
  __shared__ double sP[I][I][2], sQ[I][I][2];  // P and P^{-H} (FP64)
  __shared__ double sLogdet;
  __shared__ cpx<double> sM[(BigLane<I>::G + 1) * I * BigLane<I>::LDM];  // the P step's transposes
  // I = 3: the P step with the whole of warp 0 (k_psolve_wide's layout)
  constexpr int IW = I == 3 ? I : 1;
  __shared__ cpx<double> sWV[IW][WideP<3>::VS], sWX[IW][WideP<3>::XS], sWL[IW][WideP<3>::XS];
  __shared__ double sWRd[IW][WideP<3>::XS];
  __shared__ int sBad;

  const FastArgs& a = ra.a;
  const int p = blockIdx.x;
  const Partition& pt = a.part;
  const int n = pt.frames(p);
  const double nd = (double)n;
  const long long rlen = pt.row_len(p, a.ld), off = pt.frame_off(p), fr = pt.freq(p);
  const size_t rs = (size_t)pt.Fm * rlen;
  const C* gy = reinterpret_cast<const C*>(a.y) + (size_t)I * pt.Fm * off + fr * rlen;
  T* gv = reinterpret_cast<T*>(a.v) + (size_t)J * pt.Fm * off + fr * rlen;
  const int np = (n + 3) / 4 * 4;  // row pitch in shared memory
  C* y = reinterpret_cast<C*>(res_smem);                     // [I][np]
  T* v = reinterpret_cast<T*>(res_smem + (size_t)I * np * sizeof(C));  // [J][np]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int t = tid; t < n; t += kResThreads) {
#pragma unroll
    for (int m = 0; m < I; ++m) y[m * np + t] = gy[m * rs + t];
#pragma unroll
    for (int j = 0; j < J; ++j) v[j * np + t] = gv[j * rs + t];
  }
  if (tid < I * I) {
    const int r = tid / I, c = tid % I;
    sP[r][c][0] = a.P[((size_t)p * I * I + tid) * 2];
    sP[r][c][1] = a.P[((size_t)p * I * I + tid) * 2 + 1];
    sQ[r][c][0] = a.pinvH[((size_t)p * I * I + tid) * 2];
    sQ[r][c][1] = a.pinvH[((size_t)p * I * I + tid) * 2 + 1];
    sPT[r][c] = mk<T>((T)sP[r][c][0], (T)sP[r][c][1]);
  }
  if (tid < NA) {
    sLam[tid / I][tid % I] = a.lam[(size_t)p * NA + tid];
    sLamT[tid / I][tid % I] = (T)sLam[tid / I][tid % I];
  }
  if (tid == 0) {
    sLogdet = a.logdet[p];
    sBad = 0;
  }
  __syncthreads();

  bool singular = false;  // warp 0, lanes < I
  for (int it = 0; it < ra.iters; ++it) {
    // ---------------------------------------------------------- pass A
    {
      T acc[NVA];
#pragma unroll
      for (int q = 0; q < NVA; ++q) acc[q] = (T)0;
      // FP64: the sigmas' binary mantissas multiplied over all of the
      // thread's frames (renormalised after each frame) and their exponents
      // added; one software log2 per thread and iteration
      T lm = (T)1;
      int le = 0;
      for (int t = tid; t < n; t += kResThreads) {
        C ym[I];
#pragma unroll
        for (int m = 0; m < I; ++m) ym[m] = y[m * np + t];
        T vj[J];
#pragma unroll
        for (int j = 0; j < J; ++j) vj[j] = v[j * np + t];
        T r[I], e2[I];
#pragma unroll
        for (int i = 0; i < I; ++i) {
          C s = mk<T>(0, 0);
#pragma unroll
          for (int m = 0; m < I; ++m) cfmac(s, sPT[m][i], ym[m]);  // y~_i = sum_m conj(P_mi) y_m
          T sg = vj[0] * sLamT[0][i];
#pragma unroll
          for (int j = 1; j < J; ++j) sg = fma(vj[j], sLamT[j][i], sg);
          r[i] = recip(sg);
          e2[i] = cabs2(s);
          acc[NA] = fma(e2[i], r[i], acc[NA]);
          if constexpr (sizeof(T) == 4) {
            acc[NA + 1] += __log2f(sg);
          } else {
            int k;
            lm *= frexp(sg, &k);
            le += k;
          }
        }
        if constexpr (sizeof(T) == 8) {
          int k;
          lm = frexp(lm, &k);
          le += k;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {  // Eqs. updatev and Lambdaupdate in the form of k_estep
          T tj[I], sj = (T)0;
#pragma unroll
          for (int i = 0; i < I; ++i) {
            const T w = r[i] * fma(r[i], e2[i], (T)-1);
            tj[i] = fma(vj[j] * sLamT[j][i], w, (T)1);
            sj += tj[i];
          }
          const T rsj = recip(sj);
#pragma unroll
          for (int i = 0; i < I; ++i) acc[j * I + i] = fma(tj[i], rsj, acc[j * I + i]);
          v[j * np + t] = vj[j] * sj * (T)(1.0 / I);
        }
      }
      if constexpr (sizeof(T) == 8) acc[NA + 1] += log2(lm) + (double)le;
      ResReduce<T, NVA>::run(acc, redA, sumsA);
    }
    // the new Lambda and the problem's L2 of the entering state (FP64)
    if (tid < NA) {
      const int j = tid / I, i = tid % I;
      const double l = sLam[j][i] * ((double)I * pt.inv_n(p)) * sumsA[tid];
      if (!(l > 0.0) || !isfinite(l)) sBad = 1;
      sLam[j][i] = l;
      sLamT[j][i] = (T)l;
    } else if (tid == NA) {
      const double lf = -(double)I * nd * kLnPi + nd * sLogdet - sumsA[NA] - 0.69314718055994530942 * sumsA[NA + 1];
      if (!isfinite(lf)) sBad = 1;
      ra.hist[(size_t)it * a.F + p] = lf;
    }
    __syncthreads();
    // ---------------------------------------------------------- pass B
    // V_i for IB values of i per sub-pass: the frame's outer product y y^H
    // once, weighted by 1 / sigma_i for each i of the sub-pass
#pragma unroll 1
    for (int i0 = 0; i0 < I; i0 += IB) {
      T acc[IB * NVB];
#pragma unroll
      for (int q = 0; q < IB * NVB; ++q) acc[q] = (T)0;
      for (int t = tid; t < n; t += kResThreads) {
        C ym[I];
#pragma unroll
        for (int m = 0; m < I; ++m) ym[m] = y[m * np + t];
        T o[NVB];  // |y_r|^2, then (Re, Im) of y_r conj(y_c) for r < c
        {
          int q = I;
#pragma unroll
          for (int rr = 0; rr < I; ++rr) {
            o[rr] = cabs2(ym[rr]);
#pragma unroll
            for (int c = rr + 1; c < I; ++c) {
              o[q] = ym[rr].re * ym[c].re + ym[rr].im * ym[c].im;
              o[q + 1] = ym[rr].im * ym[c].re - ym[rr].re * ym[c].im;
              q += 2;
            }
          }
        }
#pragma unroll
        for (int ib = 0; ib < IB; ++ib) {
          const int i = i0 + ib;
          T sg = v[t] * sLamT[0][i];
#pragma unroll
          for (int j = 1; j < J; ++j) sg = fma(v[j * np + t], sLamT[j][i], sg);
          const T w = recip(sg);
#pragma unroll
          for (int q = 0; q < NVB; ++q) acc[ib * NVB + q] = fma(w, o[q], acc[ib * NVB + q]);
        }
      }
      ResReduce<T, IB * NVB>::run(acc, redB, sumsB);
      if (tid < IB * NVB) sV[i0 + tid / NVB][tid % NVB] = sumsB[tid] * pt.inv_n(p);
      __syncthreads();
    }
    // ---------------------------------------------------------- P step (warp 0)
    if constexpr (I == 3) {
      if (warp == 0) {  // lane (i, q): k_psolve_wide's factorisation, substitutions and P^{-H}
        constexpr int Q = WideP<I>::Q;
        const int i = lane % I, q = lane / I;
        const bool live = q < Q;
        for (int e = lane; e < I * NVB; e += 32) {  // V_i: the diagonal, the conjugated upper entries below it
          const int vi = e / NVB, m = e % NVB;
          if (m < I) {
            sWV[vi][m * (I + 1)] = mk(sV[vi][m], 0.0);
          } else if ((m - I) % 2 == 0) {
            int r, c;
            upper_decode<I>((m - I) / 2, r, c);
            sWV[vi][c * I + r] = mk(sV[vi][m], -sV[vi][m + 1]);
          }
        }
        if (live) sWX[i][q] = mk(sQ[q][i][0], sQ[q][i][1]);  // column i of P^{-H}
        __syncwarp();
        const bool ok = wide_ldl<I>(sWV, sWL, sWRd, i, q);
        bool sing = false;
        for (int sweep = 0; sweep < a.K; ++sweep) {
          wide_solve<I>(sWV, sWRd, sWX, i, q);
          if (sweep + 1 < a.K) {
            cpx<double> t[1];
            sing |= !(pinvh_wide<I>(sWX, i, q, t) > 0.0);
            __syncwarp();
            if (live) sWX[i][q] = t[0];
            __syncwarp();
          }
        }
        if (live) {
          const cpx<double> pv = sWX[i][q];
          sP[q][i][0] = pv.re;
          sP[q][i][1] = pv.im;
          sPT[q][i] = mk<T>((T)pv.re, (T)pv.im);
        }
        cpx<double> ph[1];
        const double det2 = pinvh_wide<I>(sWX, i, q, ph);
        if (live) {
          sQ[q][i][0] = ph[0].re;
          sQ[q][i][1] = ph[0].im;
        }
        singular |= __any_sync(0xffffffffu, !ok || sing) || !(det2 > 0.0);
        if (lane == 0) {
          sLogdet = log(det2);
          atomicAdd(a.ops, p_update_inversions(a, I));
        }
      }
    } else if (warp == 0) {
      const int g = lane / I, i = lane % I;  // problem group g = 0 is this problem; others shadow it
      cpx<double>* M = sM + (size_t)(g < BigLane<I>::G ? g : BigLane<I>::G) * I * BigLane<I>::LDM;
      double dv[I], d0[I], rd[I];
      cpx<double> lo[I * (I - 1) / 2 > 0 ? I * (I - 1) / 2 : 1];
#pragma unroll
      for (int r = 0; r < I; ++r) dv[r] = d0[r] = sV[i][r];
      {
        int m = I;
#pragma unroll
        for (int r = 0; r < I; ++r)
#pragma unroll
          for (int c = r + 1; c < I; ++c) {
            lo[lo_index(c, r)] = mk(sV[i][m], -sV[i][m + 1]);  // V_cr = conj(V_rc)
            m += 2;
          }
      }
      cpx<double> x[I];
#pragma unroll
      for (int r = 0; r < I; ++r) x[r] = mk(sQ[r][i][0], sQ[r][i][1]);  // column i of P^{-H}
      bool sing = false;
      if constexpr (I == 1) {
        sing = !(dv[0] > 0.0) || !isfinite(dv[0]);
        rd[0] = 1.0 / dv[0];
        for (int sweep = 0; sweep < a.K; ++sweep) {
          x[0] = cscale(x[0], rd[0]);
          if (sweep + 1 < a.K) pinvh_from_columns<I>(x, M, g, i, sing);
        }
      } else {
        sing = !ldl_factor<I>(dv, lo, rd);
#pragma unroll
        for (int r = 0; r < I; ++r) sing |= !(dv[r] > kCholRtol * d0[r]);
        for (int sweep = 0; sweep < a.K; ++sweep) {
          ldl_solve<I>(lo, rd, x);
          if (sweep + 1 < a.K) pinvh_from_columns<I>(x, M, g, i, sing);
        }
      }
      if (g == 0) {
#pragma unroll
        for (int r = 0; r < I; ++r) {
          sP[r][i][0] = x[r].re;
          sP[r][i][1] = x[r].im;
          sPT[r][i] = mk<T>((T)x[r].re, (T)x[r].im);
        }
      }
      const double det2 = pinvh_from_columns<I>(x, M, g, i, sing);
      if (g == 0) {
#pragma unroll
        for (int r = 0; r < I; ++r) {
          sQ[r][i][0] = x[r].re;
          sQ[r][i][1] = x[r].im;
        }
        singular |= sing;
        if (i == 0) {
          sLogdet = log(det2);
          atomicAdd(a.ops, p_update_inversions(a, I));
        }
      }
    }
    __syncthreads();
  }

  // the state back to global memory
  for (int t = tid; t < n; t += kResThreads) {
#pragma unroll
    for (int j = 0; j < J; ++j) gv[j * rs + t] = v[j * np + t];
  }
  ParamsA<T, I, J>* ta = tab_a<T, I, J>(a, p);
  if (tid < I * I) {
    const int r = tid / I, c = tid % I;
    a.P[((size_t)p * I * I + tid) * 2] = sP[r][c][0];
    a.P[((size_t)p * I * I + tid) * 2 + 1] = sP[r][c][1];
    a.pinvH[((size_t)p * I * I + tid) * 2] = sQ[r][c][0];
    a.pinvH[((size_t)p * I * I + tid) * 2 + 1] = sQ[r][c][1];
    ta->set_p(r, c, (T)sP[r][c][0], (T)sP[r][c][1]);
  }
  if (tid < NA) {
    a.lam[(size_t)p * NA + tid] = sLam[tid / I][tid % I];
    ta->set_lam(tid / I, tid % I, sLamT[tid / I][tid % I]);
  }
  if (tid == 0) {
    a.logdet[p] = sLogdet;
    if (sBad) raise_status(a.status, kDevNonfinite, p);
  }
  if (warp == 0 && lane < I && singular) raise_status(a.status, kDevSingular, p);
}

// trace[slot0 + t] = sum over the problems of hist[t][.] (fixed order).
static __global__ void __launch_bounds__(32) k_res_trace(const double* hist, int problems, double* trace, int slot0) {
  const double s = warp_sum_fixed(hist + (size_t)blockIdx.x * problems, problems);
  if (threadIdx.x == 0) trace[(slot0 + blockIdx.x) % kTraceCap] = s;
}

}  // namespace ffca
