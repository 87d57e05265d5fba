// Device helpers shared by the FastFCA-AS and FCA kernels: complex scalars,
// compensated FP32 accumulation, the balanced (f, n) work partition, the
// deterministic block reduction, and small FP64 dense solves.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ffca {

constexpr int kBlock = 256;           // threads per CTA for the streaming kernels
constexpr int kWarps = kBlock / 32;

// ------------------------------------------------------------ status words
enum DevStatus : unsigned {
  kDevOk = 0,
  kDevNonfinite = 3,
  kDevSingular = 4,
  kDevTimeout = 5,
};

// First error wins; its frequency index is kept beside it.
__device__ inline void raise_status(unsigned* status, unsigned code, int f) {
  if (atomicCAS(status, 0u, code) == 0u) status[1] = (unsigned)f;
}

// ------------------------------------------------------------ complex
template <typename T>
struct cpx {
  T re, im;
};

template <typename T>
__host__ __device__ inline cpx<T> mk(T re, T im) { return cpx<T>{re, im}; }
template <typename T>
__device__ inline cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ inline cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ inline cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename T>
__device__ inline cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename T>
__device__ inline cpx<T> cconj(cpx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ inline cpx<T> cscale(cpx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T>
__device__ inline T cabs2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += conj(a) * b
template <typename T>
__device__ inline void cfmac(cpx<T>& acc, cpx<T> a, cpx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
// acc += a * b
template <typename T>
__device__ inline void cfma(cpx<T>& acc, cpx<T> a, cpx<T> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}

// ------------------------------------------------------------ arithmetic
// Reciprocal: FP32 uses the hardware approximation refined by one
// Newton-Raphson step r <- r (2 - x r); FP64 uses the IEEE division.
__device__ inline float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * fmaf(-x, r, 2.0f);
}
__device__ inline double recip(double x) { return 1.0 / x; }
__device__ inline float logx(float x) { return __logf(x); }
__device__ inline double logx(double x) { return log(x); }

// ------------------------------------------------------------ accumulation
// Sum over frames.  FP64: plain.  FP32: Kahan-compensated (value = s - c),
// fed once per loop trip with the plain sum of that trip's few frames.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s;
  __device__ inline void zero() { s = 0.0; }
  __device__ inline void add(double x) { s += x; }
  __device__ inline double value_hi() const { return s; }
  __device__ inline double value_lo() const { return 0.0; }
};

template <>
struct Acc<float> {
  float s, c;
  __device__ inline void zero() { s = 0.f; c = 0.f; }
  __device__ inline void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  // the compensated value as an unevaluated pair (hi, lo)
  __device__ inline float value_hi() const { return s; }
  __device__ inline float value_lo() const { return -c; }
};

// Error-free sum of two floats (Knuth's TwoSum): a + b = s + e exactly.
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// Add the pair (bh, bl) into (ah, al): double-float addition.
__device__ inline void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  ah = s + e;
  al = e - (ah - s);
}

// Barrier over the threads taking part in a reduction: the whole CTA, or
// only the consumer warps of a warp-specialised CTA (named barrier 1).
template <int NTHREADS, bool NAMED>
__device__ inline void group_sync() {
  if constexpr (NAMED) {
    asm volatile("bar.sync 1, %0;" ::"n"(NTHREADS) : "memory");
  } else {
    __syncthreads();
  }
}

// Reduction of NV per-thread pairs (hi, lo) over NW warps in a fixed order.
// FP32 pairs are combined with double-float additions (compensated); FP64
// values with plain additions.  Thread t < NV writes value t (hi + lo) as a
// double to out[t].  Must be called by all NW warps.
template <typename T, int NV, int NW = kWarps, bool NAMED = false>
struct BlockReduce {
  struct Smem {
    T hi[NW][NV];
    T lo[NW][NV];
  };

  __device__ static void run(const T (&hi)[NV], const T (&lo)[NV], Smem& sm, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T h = hi[k], l = lo[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        T oh = __shfl_xor_sync(0xffffffffu, h, off);
        T ol = __shfl_xor_sync(0xffffffffu, l, off);
        combine(h, l, oh, ol);
      }
      if (lane == 0) {
        sm.hi[warp][k] = h;
        sm.lo[warp][k] = l;
      }
    }
    group_sync<32 * NW, NAMED>();
    if (threadIdx.x < NV) {
      const int k = threadIdx.x;
      T h = sm.hi[0][k], l = sm.lo[0][k];
#pragma unroll
      for (int w = 1; w < NW; ++w) combine(h, l, sm.hi[w][k], sm.lo[w][k]);
      out[k] = (double)h + (double)l;
    }
    group_sync<32 * NW, NAMED>();
  }

  __device__ static inline void combine(T& h, T& l, T oh, T ol) {
    if constexpr (sizeof(T) == 4) {
      df_add(h, l, oh, ol);
    } else {
      h += oh;
      l += ol;
    }
  }
};

// ------------------------------------------------------------ partition
// The (f, unit) plane, flattened f-major, is cut into equal contiguous
// ranges, one per CTA of a grid sized to the resident CTA count.  A CTA walks
// its range as segments of one frequency each; every frequency gets one
// partial-sum slot per CTA that touches it.
struct Partition {
  int F;             // frequencies
  int Uf;            // vector units per frequency
  long long upb;     // units per CTA
  int nblocks;       // grid size
  int max_slots;     // max CTAs touching one frequency

  __host__ __device__ inline int first_block(int f) const {
    return (int)(((long long)f * Uf) / upb);
  }
  __host__ __device__ inline int last_block(int f) const {
    return (int)(((long long)(f + 1) * Uf - 1) / upb);
  }
  __host__ __device__ inline int nslots(int f) const { return last_block(f) - first_block(f) + 1; }
};

inline Partition make_partition(int F, int Uf, int max_blocks) {
  Partition p;
  p.F = F;
  p.Uf = Uf;
  long long total = (long long)F * Uf;
  // at least one full CTA sweep of units per CTA, at most max_blocks CTAs
  long long want = (total + kBlock - 1) / kBlock;
  long long nb = want < max_blocks ? want : max_blocks;
  if (nb < 1) nb = 1;
  p.upb = (total + nb - 1) / nb;
  p.upb = (p.upb + 1) / 2 * 2;  // even: every range starts on a 16-byte boundary of v
  p.nblocks = (int)((total + p.upb - 1) / p.upb);
  if (p.nblocks < 1) p.nblocks = 1;
  // the range of one frequency spans at most ceil(Uf / upb) + 1 CTAs
  p.max_slots = (int)((Uf + p.upb - 1) / p.upb + 1);
  return p;
}

// Arrival counter: returns true in exactly one CTA, the last of `expected`
// to arrive.  Every participating thread (the CTA, or its NTHREADS consumer
// threads with NAMED) must call it after writing its partials.  Nothing
// waits on other CTAs.
template <int NTHREADS = kBlock, bool NAMED = false>
__device__ inline bool arrive_last(unsigned* counter, unsigned expected, int* flag_smem) {
  __threadfence();
  group_sync<NTHREADS, NAMED>();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    bool last = (prev == expected - 1);
    if (last) *counter = 0u;  // ready for the next launch
    *flag_smem = last ? 1 : 0;
  }
  group_sync<NTHREADS, NAMED>();
  bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

// ------------------------------------------------------------ FP64 solves
// In-place inverse of a complex I x I matrix (row-major) by Gauss-Jordan
// elimination with partial pivoting.  Also returns ln|det A|^2.  Returns
// false if a pivot is zero or not finite.
template <int I>
__device__ inline bool gj_inverse(cpx<double> (&A)[I][I], double& logabsdet2) {
  cpx<double> B[I][I];
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) B[r][c] = mk<double>(r == c ? 1.0 : 0.0, 0.0);
  logabsdet2 = 0.0;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    // pivot search in column k (rows k..I-1)
    int piv = k;
    double best = cabs2(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < I; ++r) {
      double m = cabs2(A[r][k]);
      if (m > best) { best = m; piv = r; }
    }
    if (!(best > 0.0) || !isfinite(best)) return false;
    if (piv != k) {
#pragma unroll
      for (int c = 0; c < I; ++c) {
        // swap rows k and piv with compile-time indices only
#pragma unroll
        for (int r = k + 1; r < I; ++r) {
          if (r == piv) {
            cpx<double> t = A[k][c]; A[k][c] = A[r][c]; A[r][c] = t;
            t = B[k][c]; B[k][c] = B[r][c]; B[r][c] = t;
          }
        }
      }
    }
    logabsdet2 += log(best);
    const double inv = 1.0 / best;
    const cpx<double> pinv = mk<double>(A[k][k].re * inv, -A[k][k].im * inv);  // 1 / A[k][k]
#pragma unroll
    for (int c = 0; c < I; ++c) {
      A[k][c] = cmul(A[k][c], pinv);
      B[k][c] = cmul(B[k][c], pinv);
    }
#pragma unroll
    for (int r = 0; r < I; ++r) {
      if (r == k) continue;
      const cpx<double> m = A[r][k];
#pragma unroll
      for (int c = 0; c < I; ++c) {
        A[r][c] = csub(A[r][c], cmul(m, A[k][c]));
        B[r][c] = csub(B[r][c], cmul(m, B[k][c]));
      }
    }
  }
#pragma unroll
  for (int r = 0; r < I; ++r)
#pragma unroll
    for (int c = 0; c < I; ++c) A[r][c] = B[r][c];
  return true;
}

// Solve V x = b for Hermitian positive definite V (full storage, row-major)
// by a Cholesky factorisation V = L L^H.  Returns false if V is not
// numerically positive definite: a pivot at or below kCholRtol times its
// diagonal entry (rank deficiency shows up as a pivot at rounding level).
constexpr double kCholRtol = 1e-14;

template <int I>
__device__ inline bool chol_solve(const cpx<double> (&V)[I][I], const cpx<double> (&b)[I],
                                  cpx<double> (&x)[I]) {
  cpx<double> L[I][I];
  double dinv[I];
#pragma unroll
  for (int j = 0; j < I; ++j) {
    double d = V[j][j].re;
#pragma unroll
    for (int k = 0; k < j; ++k) d -= cabs2(L[j][k]);
    if (!(d > kCholRtol * V[j][j].re) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    L[j][j] = mk<double>(ljj, 0.0);
    dinv[j] = 1.0 / ljj;
#pragma unroll
    for (int i = j + 1; i < I; ++i) {
      cpx<double> s = V[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = csub(s, cmul(L[i][k], cconj(L[j][k])));
      L[i][j] = cscale(s, dinv[j]);
    }
  }
  cpx<double> z[I];
#pragma unroll
  for (int i = 0; i < I; ++i) {  // L z = b
    cpx<double> s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = csub(s, cmul(L[i][k], z[k]));
    z[i] = cscale(s, dinv[i]);
  }
#pragma unroll
  for (int i = I - 1; i >= 0; --i) {  // L^H x = z
    cpx<double> s = z[i];
#pragma unroll
    for (int k = i + 1; k < I; ++k) s = csub(s, cmul(cconj(L[k][i]), x[k]));
    x[i] = cscale(s, dinv[i]);
  }
  return true;
}

}  // namespace ffca
