// Streaming passes of the FastFCA-AS iteration, staged through shared memory
// by the bulk-copy (TMA) engine.
//
// Each CTA is warp-specialised: one producer thread issues, per tile, one
// cp.async.bulk copy per mic row of y and per source row of v into one of
// kStages shared-memory stages (completion counted in bytes on that stage's
// "full" mbarrier); eight consumer warps wait on "full", compute from shared
// memory and release the stage on its "empty" mbarrier.  Loads are thus kept
// in flight independently of the consumers' registers.  Every wait is
// bounded; on expiry the CTA latches FFCA_ERR_TIMEOUT, stops issuing, lets
// its copies in flight land, and finishes without waiting again.
//
//   k_estep  pass A (Sec. 4.4.1): y~ = P^H y, sigma, the posterior powers
//            q_ji (Eqs. mutilde0, Phitilde0), v updated in place (Eq. updatev),
//            Lambda numerators (Eq. Lambdaupdate) and the log-likelihood
//            terms of the entering state (Eq. L2).  The last CTA to finish a
//            frequency finalises Lambda(f) and its log-likelihood; the last
//            frequency finalises the scalar.
//   k_wcov   pass B (Sec. 4.4.2): V_i(f) = (1/N) sum_n y y^H / sigma_i with
//            the new v and Lambda (Eq. FPI), into per-frequency slots.
#pragma once

#include "ffca_fastfca.cuh"

namespace ffca {

// Eight warps per CTA (seven consumers, one producer): the register file is
// split over four schedulers of 16 K registers, so two such CTAs fit an SM
// at up to 128 registers per thread, one CTA at any count.
constexpr int kConsumerWarps = 7;
constexpr int kConsumers = 32 * kConsumerWarps;
constexpr int kStreamThreads = kConsumers + 32;  // + one producer warp
constexpr int kStages = 3;

// A tile is up to T vector units of one frequency: I y rows of 16-byte units
// and J v rows of 8-byte units, contiguous in global memory per row.  T is
// one or two units per consumer thread (always even).
template <int I, int J>
struct Tile {
  static constexpr int UB = 16 * I + 8 * J;                      // bytes per unit over all rows
  static constexpr int T = (UB <= 80 ? 2 : 1) * kConsumers;      // units per tile
  static constexpr int STAGE = T * UB;                            // bytes per stage, multiple of 16
  static constexpr int SMEM = kStages * STAGE + 2 * kStages * 8;  // + mbarriers
};

// Register cap of the streaming kernels: 128 lets two CTAs share an SM where
// the per-point state fits (FP32, I <= 3, J <= 3); otherwise one CTA per SM.
template <typename T, int I, int J>
struct StreamRegs {
  static constexpr int value = (sizeof(T) == 4 && I <= 3 && J <= 3) ? 128 : 255;
};

// ------------------------------------------------------------ primitives
__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ inline void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete; gives up after ~2^31 cycles
// (about a second) or 2^26 polls, whichever comes first.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > (1ll << 31)) break;
  }
  return false;
}
// One bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0),
// completion counted on `bar`.
__device__ inline void bulk_g2s(uint32_t dst, const void* src, unsigned bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ inline void consumer_sync() { group_sync<kConsumers, true>(); }

// Walks a CTA's unit range [u0, u1) of the flattened (f, unit) plane as
// tiles of at most T units that never cross a frequency.
struct TileIter {
  long long u, u1;
  int Uf, T;
  int f, k, n;
  bool seg_end;
  __device__ TileIter(long long u0_, long long u1_, int Uf_, int T_) : u(u0_), u1(u1_), Uf(Uf_), T(T_) {}
  __device__ bool next() {
    if (u >= u1) return false;
    f = (int)(u / Uf);
    k = (int)(u - (long long)f * Uf);
    const int kend = (int)min((long long)Uf, k + (u1 - u));
    n = min(T, kend - k);
    seg_end = (k + n == kend);
    u += n;
    return true;
  }
};

struct Pipe {
  unsigned char* smem;
  uint32_t bars;  // full[s] at bars + 8 s, empty[s] at bars + 8 (kStages + s)
  __device__ uint32_t full(int s) const { return bars + 8 * s; }
  __device__ uint32_t empty(int s) const { return bars + 8 * (kStages + s); }
};

// Producer: one thread.  y units are 16 bytes, v units 8 bytes; ranges start
// on even units, so every copy is 16-byte aligned and a multiple of 16 bytes.
template <int I, int J>
__device__ void produce(const FastArgs& a, const Pipe& pp, long long u0, long long u1, long long row,
                        volatile int* abort) {
  using TC = Tile<I, J>;
  const char* y = static_cast<const char*>(a.y);
  const char* v = static_cast<const char*>(a.v);
  TileIter it(u0, u1, a.part.Uf, TC::T);
  int t = 0;
  while (it.next()) {
    const int s = t % kStages;
    if (t >= kStages && !*abort && !mbar_wait(pp.empty(s), ((t / kStages) - 1) & 1)) {
      raise_status(a.status, kDevTimeout, it.f);
      *abort = 1;
    }
    if (*abort) break;
    const uint32_t st = smem_u32(pp.smem + (size_t)s * TC::STAGE);
    mbar_expect_tx(pp.full(s), (unsigned)it.n * TC::UB);
#pragma unroll
    for (int m = 0; m < I; ++m)
      bulk_g2s(st + m * TC::T * 16, y + (((size_t)m * a.F + it.f) * row + it.k) * 16,
               (unsigned)it.n * 16, pp.full(s));
#pragma unroll
    for (int j = 0; j < J; ++j)
      bulk_g2s(st + I * TC::T * 16 + j * TC::T * 8, v + (((size_t)j * a.F + it.f) * row + it.k) * 8,
               (unsigned)it.n * 8, pp.full(s));
    ++t;
  }
  // let the copies of the last stages land before this thread leaves
  for (int d = t > kStages ? t - kStages : 0; d < t; ++d) mbar_wait(pp.full(d % kStages), (d / kStages) & 1);
}

__device__ inline Pipe setup_pipe(unsigned char* smem, int stage_bytes, volatile int* abort) {
  Pipe pp;
  pp.smem = smem;
  pp.bars = smem_u32(smem + (size_t)kStages * stage_bytes);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(pp.full(s), 1);
      mbar_init(pp.empty(s), kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort = 0;
  }
  __syncthreads();
  return pp;
}

// Consumer side of one tile: wait for it unless the CTA has given up.
__device__ inline bool consumer_acquire(const FastArgs& a, const Pipe& pp, int t, int f, volatile int* abort) {
  if (*abort) return false;
  if (mbar_wait(pp.full(t % kStages), (t / kStages) & 1)) return true;
  raise_status(a.status, kDevTimeout, f);
  *abort = 1;
  return false;
}
__device__ inline void consumer_release(const Pipe& pp, int t) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(pp.empty(t % kStages));
}

// -------------------------------------------------------------- pass A
template <typename T, int I, int J, bool UPDATE>
__global__ void __maxnreg__((StreamRegs<T, I, J>::value)) k_estep(FastArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using TC = Tile<I, J>;
  using Red = BlockReduce<T, (UPDATE ? J * I + 1 : 1), kConsumerWarps, true>;
  constexpr int FU = Vec<T>::FU;
  constexpr int NV = UPDATE ? J * I + 1 : 1;  // Lambda numerators, then loglik
  constexpr int LL = NV - 1;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ typename Red::Smem red;
  __shared__ double sP[I][I][2];
  __shared__ double sLam[J][I];
  __shared__ int sflag;
  __shared__ int sabort;
  volatile int* abort = &sabort;

  const Partition pt = a.part;
  const long long total = (long long)pt.F * pt.Uf;
  const long long u0 = (long long)blockIdx.x * pt.upb;
  const long long u1 = min(u0 + pt.upb, total);
  const long long row = a.ld / FU;  // vector units per (mic or source, f) row
  const Pipe pp = setup_pipe(smem, TC::STAGE, abort);

  if (threadIdx.x >= kConsumers) {
    if (threadIdx.x == kConsumers) produce<I, J>(a, pp, u0, u1, row, abort);
    return;
  }

  VV* __restrict__ vg = reinterpret_cast<VV*>(a.v);
  const int tid = threadIdx.x;
  cpx<T> Pc[I][I];  // P(f): y~_i = sum_m conj(P_mi) y_m
  T lam[J][I], ilam[J][I];
  Acc<T> acc[NV];

  TileIter it(u0, u1, pt.Uf, TC::T);
  bool seg_new = true;
  for (int t = 0; it.next(); ++t) {
    const int f = it.f;
    if (seg_new) {
      consumer_sync();  // the previous segment is done with sP / sLam
      if (tid < I * I) {
        sP[tid / I][tid % I][0] = a.P[((size_t)f * I * I + tid) * 2];
        sP[tid / I][tid % I][1] = a.P[((size_t)f * I * I + tid) * 2 + 1];
      }
      if (tid < J * I) sLam[tid / I][tid % I] = a.lam[(size_t)f * J * I + tid];
      consumer_sync();
#pragma unroll
      for (int r = 0; r < I; ++r)
#pragma unroll
        for (int c = 0; c < I; ++c) Pc[r][c] = mk<T>((T)sP[r][c][0], (T)sP[r][c][1]);
#pragma unroll
      for (int j = 0; j < J; ++j)
#pragma unroll
        for (int i = 0; i < I; ++i) {
          lam[j][i] = (T)sLam[j][i];
          ilam[j][i] = recip(lam[j][i]);
        }
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q].zero();
      seg_new = false;
    }

    if (consumer_acquire(a, pp, t, f, abort)) {
      const unsigned char* st = pp.smem + (size_t)(t % kStages) * TC::STAGE;
      const VY* ys = reinterpret_cast<const VY*>(st);
      const VV* vs = reinterpret_cast<const VV*>(st + I * TC::T * 16);
      T grp[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) grp[q] = (T)0;
#pragma unroll 1
      for (int q = tid; q < it.n; q += kConsumers) {
        VY yu[I];
        VV vu[J];
#pragma unroll
        for (int m = 0; m < I; ++m) yu[m] = ys[m * TC::T + q];
#pragma unroll
        for (int j = 0; j < J; ++j) vu[j] = vs[j * TC::T + q];
        const int k = it.k + q;
#pragma unroll
        for (int e = 0; e < FU; ++e) {
          if (k * FU + e >= a.N) continue;
          cpx<T> yt[I];
#pragma unroll
          for (int i = 0; i < I; ++i) {
            cpx<T> s = mk<T>(0, 0);
#pragma unroll
            for (int m = 0; m < I; ++m) cfmac(s, Pc[m][i], yframe(yu[m], e));
            yt[i] = s;
          }
          T vv[J];
#pragma unroll
          for (int j = 0; j < J; ++j) vv[j] = vframe(vu[j], e);
          T rs[I], e2[I];
          T ll = (T)0;
#pragma unroll
          for (int i = 0; i < I; ++i) {
            T s = vv[0] * lam[0][i];
#pragma unroll
            for (int j = 1; j < J; ++j) s = fma(vv[j], lam[j][i], s);
            rs[i] = recip(s);
            e2[i] = cabs2(yt[i]);
            ll += logx(s) + e2[i] * rs[i];
          }
          grp[LL] += ll;
          if constexpr (UPDATE) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
              T qv[I];
              T vn = (T)0;
#pragma unroll
              for (int i = 0; i < I; ++i) {
                const T aji = vv[j] * lam[j][i];          // v_j [Lambda_j]_ii
                const T g = aji * rs[i];                   // Wiener gain
                const T phi = fma(-aji, g, aji);           // Eq. Phitilde0
                qv[i] = fma(g * g, e2[i], phi);            // |mu~|^2 + phi~
                vn = fma(qv[i], ilam[j][i], vn);
              }
              vn *= (T)(1.0 / I);                          // Eq. updatev
              vset(vu[j], e, vn);
              const T rv = recip(vn);
#pragma unroll
              for (int i = 0; i < I; ++i) grp[j * I + i] = fma(qv[i], rv, grp[j * I + i]);
            }
          }
        }
        if constexpr (UPDATE) {
#pragma unroll
          for (int j = 0; j < J; ++j) vg[((size_t)j * pt.F + f) * row + k] = vu[j];
        }
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q].add(grp[q]);
    }
    consumer_release(pp, t);

    if (it.seg_end) {
      T hi[NV], lo[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        hi[q] = acc[q].value_hi();
        lo[q] = acc[q].value_lo();
      }
      const int slot = (int)blockIdx.x - pt.first_block(f);
      Red::run(hi, lo, red, a.part_buf + ((size_t)f * pt.max_slots + slot) * NV);
      if (arrive_last<kConsumers, true>(a.cnt + f, (unsigned)pt.nslots(f), &sflag)) {
        if (tid < NV) {
          const double tot = sum_slots(a.part_buf, f, pt.nslots(f), pt.max_slots, NV, tid);
          if (tid == LL) {
            const double lf = -(double)I * a.N * kLnPi + (double)a.N * __ldcg(a.logdet + f) - tot;
            if (!isfinite(lf)) raise_status(a.status, kDevNonfinite, f);
            a.llf[f] = lf;
          } else {
            const double lnew = tot / a.N;  // Eq. Lambdaupdate
            if (!(lnew > 0.0) || !isfinite(lnew)) raise_status(a.status, kDevNonfinite, f);
            a.lam[(size_t)f * J * I + tid] = lnew;
          }
        }
        if (arrive_last<kConsumers, true>(a.gcnt, (unsigned)pt.F, &sflag)) finalize_trace(a);
      }
      seg_new = true;
    }
  }
}

// -------------------------------------------------------------- pass B
template <typename T, int I, int J>
__global__ void __maxnreg__((StreamRegs<T, I, J>::value)) k_wcov(FastArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using TC = Tile<I, J>;
  constexpr int FU = Vec<T>::FU;
  constexpr int I2 = I * I;
  constexpr int NV = I * I2;
  using Red = BlockReduce<T, NV, kConsumerWarps, true>;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ typename Red::Smem red;
  __shared__ double sLam[J][I];
  __shared__ int sabort;
  volatile int* abort = &sabort;

  const Partition pt = a.part;
  const long long total = (long long)pt.F * pt.Uf;
  const long long u0 = (long long)blockIdx.x * pt.upb;
  const long long u1 = min(u0 + pt.upb, total);
  const long long row = a.ld / FU;
  const Pipe pp = setup_pipe(smem, TC::STAGE, abort);

  if (threadIdx.x >= kConsumers) {
    if (threadIdx.x == kConsumers) produce<I, J>(a, pp, u0, u1, row, abort);
    return;
  }

  const int tid = threadIdx.x;
  T lam[J][I];
  // Per-thread sums over this segment's frames (a few dozen at most at full
  // size); the tree across threads is compensated.
  T acc[NV];

  TileIter it(u0, u1, pt.Uf, TC::T);
  bool seg_new = true;
  for (int t = 0; it.next(); ++t) {
    const int f = it.f;
    if (seg_new) {
      consumer_sync();
      if (tid < J * I) sLam[tid / I][tid % I] = a.lam[(size_t)f * J * I + tid];
      consumer_sync();
#pragma unroll
      for (int j = 0; j < J; ++j)
#pragma unroll
        for (int i = 0; i < I; ++i) lam[j][i] = (T)sLam[j][i];
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = (T)0;
      seg_new = false;
    }

    if (consumer_acquire(a, pp, t, f, abort)) {
      const unsigned char* st = pp.smem + (size_t)(t % kStages) * TC::STAGE;
      const VY* ys = reinterpret_cast<const VY*>(st);
      const VV* vs = reinterpret_cast<const VV*>(st + I * TC::T * 16);
#pragma unroll 1
      for (int q = tid; q < it.n; q += kConsumers) {
        VY yu[I];
        VV vu[J];
#pragma unroll
        for (int m = 0; m < I; ++m) yu[m] = ys[m * TC::T + q];
#pragma unroll
        for (int j = 0; j < J; ++j) vu[j] = vs[j * TC::T + q];
        const int k = it.k + q;
#pragma unroll
        for (int e = 0; e < FU; ++e) {
          if (k * FU + e >= a.N) continue;
          cpx<T> ym[I];
#pragma unroll
          for (int m = 0; m < I; ++m) ym[m] = yframe(yu[m], e);
          T w[I];
#pragma unroll
          for (int i = 0; i < I; ++i) {
            T s = vframe(vu[0], e) * lam[0][i];
#pragma unroll
            for (int j = 1; j < J; ++j) s = fma(vframe(vu[j], e), lam[j][i], s);
            w[i] = recip(s);
          }
          // y y^H, packed: diagonal |y_r|^2, then y_r conj(y_c) for r < c
          T pk[I2];
          int m = I;
#pragma unroll
          for (int r = 0; r < I; ++r) {
            pk[r] = cabs2(ym[r]);
#pragma unroll
            for (int c = r + 1; c < I; ++c) {
              pk[m] = fma(ym[r].re, ym[c].re, ym[r].im * ym[c].im);
              pk[m + 1] = fma(ym[r].im, ym[c].re, -ym[r].re * ym[c].im);
              m += 2;
            }
          }
#pragma unroll
          for (int i = 0; i < I; ++i)
#pragma unroll
            for (int mm = 0; mm < I2; ++mm) acc[i * I2 + mm] = fma(w[i], pk[mm], acc[i * I2 + mm]);
        }
      }
    }
    consumer_release(pp, t);

    if (it.seg_end) {
      T lo[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) lo[q] = (T)0;
      const int slot = (int)blockIdx.x - pt.first_block(f);
      Red::run(acc, lo, red, a.part_buf + ((size_t)f * pt.max_slots + slot) * NV);
      seg_new = true;
    }
  }
}

}  // namespace ffca
