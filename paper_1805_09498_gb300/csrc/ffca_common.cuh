// Device helpers shared by the FastFCA-AS and FCA kernels: complex scalars,
// compensated FP32 accumulation (Kahan sums, double-float pair sums), the
// balanced (f, n) work partition, the deterministic block reduction, and
// small FP64 dense solves.
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
__host__ __device__ inline cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ inline cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ inline cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename T>
__host__ __device__ inline cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename T>
__host__ __device__ inline cpx<T> cconj(cpx<T> a) { return {a.re, -a.im}; }
template <typename T>
__host__ __device__ inline cpx<T> cscale(cpx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T>
__host__ __device__ inline T cabs2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
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
// FP64: the hardware estimate refined by two Newton-Raphson steps
// r <- r + r (1 - x r) (each step doubles the correct bits; the result is
// within an ulp or two of 1/x, not correctly rounded).  Zero, infinite and
// subnormal x give a non-finite result, which the kernels report.
__device__ inline double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ inline float logx(float x) { return __logf(x); }
__device__ inline double logx(double x) { return log(x); }

// ------------------------------------------------------------ accumulation
// Compensated (Kahan) sum over frames in FP32 held in two floats: h, the
// running total, and p, the partial of the frames added since the last fold,
// which starts from the rounding error the previous fold left behind.  Frames
// are added to p (a few per fold: the units a thread takes from a few tiles);
// fold() is one Kahan step, h + p = t exactly up to the error e it returns in
// p (t = h + p, e = p - (t - h)), so that the error of the whole sum is that
// of the short partials plus O(u^2) terms, independent of the number of
// frames.  The two floats take the registers of the packed pair that held a
// plain sum per frame lane.  value() is the compensated total.
struct KSum {
  float h, p;
  __device__ inline void zero() { h = 0.f; p = 0.f; }
  __device__ inline void add(float x) { p += x; }
  __device__ inline void fold() {
    const float t = __fadd_rn(h, p);
    p = __fsub_rn(p, __fsub_rn(t, h));
    h = t;
  }
  __device__ inline float value() const { return __fadd_rn(h, p); }
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

// Reduction of NV per-thread pairs (hi, lo) over NW warps, for larger NV: a
// butterfly reduce-scatter inside each warp (at level `off` every lane keeps
// half of its remaining values and receives the partner's partial sums of
// that half from lane ^ off), so that 31 exchanges reduce 32 values where a
// tree per value needs 5 each; lane l ends with value l of its chunk.  The
// NW warp results are then summed in shared memory in warp order.  FP32
// pairs combine with double-float additions, FP64 values plainly.  Thread
// t < NV writes value t to out[t] (as a double).  Called by all NW warps.
template <typename T, int NV, int NW, bool NAMED>
struct ButterflyReduce {
  static constexpr int NC = (NV + 31) / 32;  // chunks of 32 values
  static constexpr bool PAIR = sizeof(T) == 4;
  struct Smem {
    T hi[NW][NC * 32];
    T lo[PAIR ? NW : 1][PAIR ? NC * 32 : 1];
  };

  __device__ static void run(const T (&hi)[NV], const T (&lo)[NV], Smem& sm, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T h[32], l[32];
#pragma unroll
      for (int v = 0; v < 32; ++v) {
        const int idx = c * 32 + v;
        h[v] = idx < NV ? hi[idx] : (T)0;
        l[v] = idx < NV ? lo[idx] : (T)0;
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
          T kh = up ? h[j + off] : h[j];
          const T sh = up ? h[j] : h[j + off];
          const T rh = __shfl_xor_sync(0xffffffffu, sh, off);
          if constexpr (PAIR) {
            T kl = up ? l[j + off] : l[j];
            const T sl = up ? l[j] : l[j + off];
            const T rl = __shfl_xor_sync(0xffffffffu, sl, off);
            df_add(kh, kl, rh, rl);
            l[j] = kl;
          } else {
            kh += rh;
          }
          h[j] = kh;
        }
      }
      sm.hi[warp][c * 32 + lane] = h[0];
      if constexpr (PAIR) sm.lo[warp][c * 32 + lane] = l[0];
    }
    group_sync<32 * NW, NAMED>();
    for (int t = threadIdx.x; t < NV; t += 32 * NW) {
      T h = sm.hi[0][t];
      T l = PAIR ? sm.lo[0][t] : (T)0;
#pragma unroll
      for (int w = 1; w < NW; ++w) {
        if constexpr (PAIR) {
          df_add(h, l, sm.hi[w][t], sm.lo[w][t]);
        } else {
          h += sm.hi[w][t];
        }
      }
      out[t] = (double)h + (double)l;
    }
    group_sync<32 * NW, NAMED>();
  }
};

// ------------------------------------------------------------ partition
// Work is a list of independent problems, one per (mixture, frequency): the
// problem's units (16-byte vector units of its frames) are contiguous in the
// flattened unit space.  A single mixture is the uniform case (problem p =
// frequency p, every problem N frames and Uf units, no tables); a batch of
// mixtures of uneven length passes per-problem tables.  The unit space is
// cut into equal contiguous ranges, one per CTA (or pipeline group) of a
// grid sized to what is resident at once.  A CTA walks its range as segments
// of one problem each; every problem gets one partial-sum slot per CTA that
// touches it.
struct ProbInfo {
  long long frame_off;  // sum of the row lengths of the earlier mixtures (multiple of 4): the
                        // mixture's y block [I][Fm][ld] starts at frame I Fm frame_off, its v
                        // block [J][Fm][ld] at J Fm frame_off
  int f;                // frequency: the problem's rows are [mic or source][f] of its block
  int n;                // frames
  double inv_n;         // 1 / n
  int ld;               // row length of the mixture's blocks (multiple of 4, >= n)
};

struct Partition {
  int F;                    // problems
  int Fm;                   // frequencies per mixture (row addressing)
  int Uf;                   // uniform case: vector units per problem
  int N;                    // uniform case: frames per problem
  double inv_n_uniform;     // uniform case: 1 / N
  const ProbInfo* info;     // ragged case: [F] (nullptr in the uniform case)
  const long long* ustart;  // ragged case: [F + 1] first unit of each problem
  const long long* bstart;  // ragged case: [nblocks + 1] first unit of each CTA's range
  const int2* slots;        // ragged case: [F] (first CTA, CTAs) touching each problem
  long long total;          // units
  long long upb;            // uniform case: units per CTA
  int nblocks;              // CTAs (pipeline groups) of the grid
  int max_slots;            // max CTAs touching one problem

  __host__ __device__ inline long long start(int p) const { return ustart ? ustart[p] : (long long)p * Uf; }
  __host__ __device__ inline int units(int p) const { return (int)(start(p + 1) - start(p)); }
  // the unit range [block_start(b), block_start(b + 1)) of CTA b (empty for b >= nblocks)
  __device__ inline long long block_start(int b) const {
    if (b >= nblocks) return total;
    return bstart ? bstart[b] : min((long long)b * upb, total);
  }
  __device__ inline int first_block(int p) const { return slots ? slots[p].x : (int)(start(p) / upb); }
  __device__ inline int nslots(int p) const {
    return slots ? slots[p].y : (int)((start(p + 1) - 1) / upb) - (int)(start(p) / upb) + 1;
  }
  __device__ inline int freq(int p) const { return info ? info[p].f : p; }
  __device__ inline int frames(int p) const { return info ? info[p].n : N; }
  __device__ inline long long frame_off(int p) const { return info ? info[p].frame_off : 0; }
  // row length (frames) of problem p's blocks; ld_uniform in the uniform case
  __device__ inline long long row_len(int p, long long ld_uniform) const { return info ? info[p].ld : ld_uniform; }
  __device__ inline double inv_n(int p) const { return info ? info[p].inv_n : inv_n_uniform; }
  // the problem that holds unit u (0 <= u < total)
  __device__ inline int problem_of(long long u) const {
    if (!ustart) return (int)(u / Uf);
    int lo = 0, hi = F - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (ustart[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
};

inline void finish_partition(Partition& p, int max_blocks) {
  // at least one full CTA sweep of units per CTA, at most max_blocks CTAs
  long long want = (p.total + kBlock - 1) / kBlock;
  long long nb = want < max_blocks ? want : max_blocks;
  if (nb < 1) nb = 1;
  p.upb = (p.total + nb - 1) / nb;
  p.upb = (p.upb + 1) / 2 * 2;  // even: every range starts on a 16-byte boundary of v
  if (p.upb < 2) p.upb = 2;
  p.nblocks = (int)((p.total + p.upb - 1) / p.upb);
  if (p.nblocks < 1) p.nblocks = 1;
}

// Uniform problems: F of Uf units and N frames each.
inline Partition make_partition(int F, int Uf, int max_blocks, int N = 0) {
  Partition p;
  p.F = F;
  p.Fm = F;
  p.Uf = Uf;
  p.N = N;
  p.inv_n_uniform = N > 0 ? 1.0 / N : 0.0;
  p.info = nullptr;
  p.ustart = nullptr;
  p.bstart = nullptr;
  p.slots = nullptr;
  p.total = (long long)F * Uf;
  finish_partition(p, max_blocks);
  // the range of one problem spans at most ceil(Uf / upb) + 1 CTAs
  p.max_slots = (int)((Uf + p.upb - 1) / p.upb + 1);
  return p;
}

// Ragged problems: ustart_host [F + 1] (host copy of the unit starts).  A
// CTA's time is its units plus a fixed cost per problem it touches (the
// segment's reduction and parameter hand-over), so the CTA ranges balance
// cost = units + seg_cost per problem, not units alone: a run of short
// problems gets fewer units.  Fills bstart_host [nblocks + 1] and
// slots_host [F]; the device copies are attached by the caller.
inline Partition make_partition_ragged(int F, int Fm, const long long* ustart_host, int max_blocks,
                                       long long seg_cost, long long* bstart_host, int2* slots_host) {
  Partition p;
  p.F = F;
  p.Fm = Fm;
  p.Uf = 0;
  p.N = 0;
  p.inv_n_uniform = 0.0;
  p.info = nullptr;
  p.ustart = nullptr;
  p.bstart = nullptr;
  p.slots = nullptr;
  p.total = ustart_host[F];
  finish_partition(p, max_blocks);
  const int nb = p.nblocks;
  // boundaries at equal steps of the cumulative cost, rounded down to even
  // units, strictly increasing (every range non-empty)
  const double C = (double)p.total + (double)seg_cost * F;
  bstart_host[0] = 0;
  int q = 0;
  for (int b = 1; b < nb; ++b) {
    const double x = C * b / nb;
    while (q + 1 < F && (double)ustart_host[q + 1] + (double)seg_cost * (q + 1) <= x) ++q;
    const double within = x - ((double)ustart_host[q] + (double)seg_cost * q) - (double)seg_cost;
    long long u = ustart_host[q] + (within > 0.0 ? (long long)within : 0);
    if (u > ustart_host[q + 1]) u = ustart_host[q + 1];
    u = u / 2 * 2;
    const long long lo = bstart_host[b - 1] + 2, hi = p.total - 2LL * (nb - b);
    bstart_host[b] = u < lo ? lo : (u > hi ? hi : u);
  }
  bstart_host[nb] = p.total;
  // first CTA and number of CTAs touching each problem
  int b = 0, ms = 1;
  for (int r = 0; r < F; ++r) {
    while (bstart_host[b + 1] <= ustart_host[r]) ++b;
    int e = b;
    while (bstart_host[e + 1] < ustart_host[r + 1]) ++e;
    slots_host[r] = make_int2(b, e - b + 1);
    if (e - b + 1 > ms) ms = e - b + 1;
  }
  p.max_slots = ms;
  return p;
}

// Arrival counter: returns true in exactly one CTA, the last of `expected`
// to arrive.  Every participating thread (the CTA, or its NTHREADS consumer
// threads with NAMED) must call it; the threads below `writers` (those that
// wrote data the last CTA will read) fence their writes first.  Nothing
// waits on other CTAs.
template <int NTHREADS = kBlock, bool NAMED = false>
__device__ inline bool arrive_last(unsigned* counter, unsigned expected, int* flag_smem,
                                   int writers = NTHREADS) {
  if ((int)threadIdx.x < writers) __threadfence();
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
// Determinant of the (I-1) x (I-1) minor of the complex I x I matrix A that
// leaves out row r and column c (I <= 4).
template <int I>
__host__ __device__ inline cpx<double> minor_det(const cpx<double> (&A)[I][I], int r, int c) {
  if constexpr (I == 1) {
    return mk(1.0, 0.0);
  } else {
    int rows[I - 1], cols[I - 1];
#pragma unroll
    for (int k = 0, nr = 0, nc = 0; k < I; ++k) {
      if (k != r) rows[nr++] = k;
      if (k != c) cols[nc++] = k;
    }
    if constexpr (I == 2) {
      return A[rows[0]][cols[0]];
    } else if constexpr (I == 3) {
      return csub(cmul(A[rows[0]][cols[0]], A[rows[1]][cols[1]]), cmul(A[rows[0]][cols[1]], A[rows[1]][cols[0]]));
    } else {
      static_assert(I == 4, "I <= 4");
      auto e = [&](int rr, int cc) { return A[rows[rr]][cols[cc]]; };
      cpx<double> d = cmul(e(0, 0), csub(cmul(e(1, 1), e(2, 2)), cmul(e(1, 2), e(2, 1))));
      d = csub(d, cmul(e(0, 1), csub(cmul(e(1, 0), e(2, 2)), cmul(e(1, 2), e(2, 0)))));
      return cadd(d, cmul(e(0, 2), csub(cmul(e(1, 0), e(2, 1)), cmul(e(1, 1), e(2, 0)))));
    }
  }
}

// Column i of the cofactor matrix of A: C_ri, r = 0..I-1.  Expanding the
// determinant along column i gives det A = sum_r A_ri C_ri, and row i of the
// inverse is (A^{-1})_ir = C_ri / det A.
template <int I>
__host__ __device__ inline cpx<double> column_cofactors(const cpx<double> (&A)[I][I], int i, cpx<double> (&C)[I]) {
  cpx<double> det = mk(0.0, 0.0);
#pragma unroll
  for (int r = 0; r < I; ++r) {
    const cpx<double> m = minor_det<I>(A, r, i);
    C[r] = ((r + i) & 1) ? mk(-m.re, -m.im) : m;
    det = cadd(det, cmul(A[r][i], C[r]));
  }
  return det;
}

// 2 x 2 minors of the row pair (r0, r1) of a complex 4 x 4 matrix, for the
// six column pairs in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
__host__ __device__ inline void pair_minors4(const cpx<double> (&A)[4][4], int r0, int r1, cpx<double> (&m)[6]) {
  int k = 0;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = p + 1; q < 4; ++q) m[k++] = csub(cmul(A[r0][p], A[r1][q]), cmul(A[r0][q], A[r1][p]));
}
// index of the column pair (p, q), p < q, in that order
__host__ __device__ constexpr int pair_index4(int p, int q) { return p == 0 ? q - 1 : (p == 1 ? q + 1 : 5); }

// Determinant and full cofactor matrix of a complex I x I matrix with
// compile-time indexing only (registers, no local memory), C_rc =
// (-1)^(r+c) minor_rc, so that A^{-1} = C^T / det A.  I <= 3: every minor
// directly.  I = 4: Laplace expansion by the row pairs (0,1) and (2,3): with
// s the 2 x 2 minors of rows 0-1 and t those of rows 2-3, the 3 x 3 minor
// leaving out row r and column c (other columns p < q < w) expands along the
// remaining row of the other pair, e.g. minor_0c = A_1p t_qw - A_1q t_pw +
// A_1w t_pq, and det A = sum over complementary column pairs of
// +-s_pq t_(rest); 12 + 48 + 6 complex products instead of 16 separate 3 x 3
// determinants.
template <int I>
__host__ __device__ inline cpx<double> cofactors(const cpx<double> (&A)[I][I], cpx<double> (&C)[I][I]) {
  if constexpr (I == 4) {
    cpx<double> s[6], t[6];
    pair_minors4(A, 0, 1, s);
    pair_minors4(A, 2, 3, t);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int p = c == 0 ? 1 : 0, q = c <= 1 ? 2 : 1, w = c == 3 ? 2 : 3;  // the other columns
      const int iqw = pair_index4(q, w), ipw = pair_index4(p, w), ipq = pair_index4(p, q);
      // rows 0 / 1 left out: expand along row 1 / 0 with the bottom minors
      // rows 2 / 3 left out: expand along row 3 / 2 with the top minors
      const int src[4] = {1, 0, 3, 2};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const cpx<double>* m = r < 2 ? t : s;
        const int b = src[r];
        cpx<double> d = cmul(A[b][p], m[iqw]);
        d = csub(d, cmul(A[b][q], m[ipw]));
        d = cadd(d, cmul(A[b][w], m[ipq]));
        C[r][c] = ((r + c) & 1) ? mk(-d.re, -d.im) : d;
      }
    }
    // det = s01 t23 - s02 t13 + s03 t12 + s12 t03 - s13 t02 + s23 t01
    cpx<double> det = cmul(s[0], t[5]);
    det = csub(det, cmul(s[1], t[4]));
    det = cadd(det, cmul(s[2], t[3]));
    det = cadd(det, cmul(s[3], t[2]));
    det = csub(det, cmul(s[4], t[1]));
    return cadd(det, cmul(s[5], t[0]));
  } else {
#pragma unroll
    for (int r = 0; r < I; ++r)
#pragma unroll
      for (int c = 0; c < I; ++c) {
        const cpx<double> m = minor_det<I>(A, r, c);
        C[r][c] = ((r + c) & 1) ? mk(-m.re, -m.im) : m;
      }
    cpx<double> det = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < I; ++c) det = cadd(det, cmul(A[0][c], C[0][c]));
    return det;
  }
}

// Determinant alone (the same expansions).
template <int I>
__host__ __device__ inline cpx<double> determinant(const cpx<double> (&A)[I][I]) {
  if constexpr (I == 4) {
    cpx<double> s[6], t[6];
    pair_minors4(A, 0, 1, s);
    pair_minors4(A, 2, 3, t);
    cpx<double> det = cmul(s[0], t[5]);
    det = csub(det, cmul(s[1], t[4]));
    det = cadd(det, cmul(s[2], t[3]));
    det = cadd(det, cmul(s[3], t[2]));
    det = csub(det, cmul(s[4], t[1]));
    return cadd(det, cmul(s[5], t[0]));
  } else {
    cpx<double> det = mk(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < I; ++c) {
      const cpx<double> m = minor_det<I>(A, 0, c);
      det = cadd(det, cmul(A[0][c], (c & 1) ? mk(-m.re, -m.im) : m));
    }
    return det;
  }
}

// Relative threshold below which a positive definite determinant or pivot is
// treated as rank deficient (rounding level in FP64).
constexpr double kCholRtol = 1e-14;

}  // namespace ffca
