// Streaming passes of the FastFCA-AS iteration, staged through shared memory
// by the bulk-copy (TMA) engine.
//
// Each CTA runs one or two independent warp-specialised pipelines ("groups"),
// each working through its own contiguous range of the (f, unit) plane (a
// "virtual block" of the partition).  In a group one producer thread issues,
// per tile, one cp.async.bulk copy per mic row of y and per source row of v
// into one of kStages shared-memory stages (completion counted in bytes on
// that stage's "full" mbarrier); seven consumer warps wait on "full", compute
// from shared memory and release the stage on its "empty" mbarrier.  Loads
// are thus kept in flight independently of the consumers' registers.  The
// groups share one CTA (rather than being two CTAs per SM) because the warp
// scheduler favours the warps of the CTA launched first: with separate CTAs
// of equal work the second one finished ~15% later.  Group membership is
// interleaved over warp indices so that every scheduler hosts both groups.
// Every wait is bounded; on expiry the group latches FFCA_ERR_TIMEOUT, stops
// issuing, lets its copies in flight land, and finishes without waiting.
//
//   k_estep  pass A (Sec. 4.4.1): y~ = P^H y, sigma, the posterior powers
//            q_ji (Eqs. mutilde0, Phitilde0), v updated in place (Eq. updatev),
//            Lambda numerators (Eq. Lambdaupdate) and the log-likelihood
//            terms of the entering state (Eq. L2), into per-frequency slots
//            (finalised by k_afinal).
//   k_wcov   pass B (Sec. 4.4.2): V_i(f) = (1/N) sum_n y y^H / sigma_i with
//            the new v and Lambda (Eq. FPI), into per-frequency slots
//            (finalised by k_psolve).
// Neither kernel loads anything but its tiles: the per-frequency parameters
// ride along in each stage, so no consumer waits on global memory.
#pragma once

#include <type_traits>

#include "ffca_fastfca.cuh"

namespace ffca {

// Two groups of eight warps (seven consumers, one producer) per CTA: the
// register file is split over four schedulers of 16 K registers, so the 16
// warps fit at up to 128 registers per thread.
#ifndef FFCA_CONSUMER_WARPS
#define FFCA_CONSUMER_WARPS 7
#endif

// Stages per pipeline: as many as the shared-memory budget holds, at most
// FFCA_MAX_STAGES (the bytes in flight per SM must cover the DRAM latency).
#ifndef FFCA_MAX_STAGES
#define FFCA_MAX_STAGES 8
#endif
#ifndef FFCA_TILE_UNITS_PER_THREAD
#define FFCA_TILE_UNITS_PER_THREAD 2
#endif
constexpr int kConsumerWarps = FFCA_CONSUMER_WARPS;
constexpr int kConsumers = 32 * kConsumerWarps;
constexpr int kGroupWarps = kConsumerWarps + 1;  // + one producer warp
constexpr int kGroupThreads = 32 * kGroupWarps;
constexpr int kStreamSmemBudget = 200 * 1024;    // dynamic shared memory per CTA
static_assert(kGroupWarps % 4 == 0, "groups interleave in units of four warps");

// Pipelines per CTA: two (at most FFCA_MAX_GROUPS) where the per-point state
// fits 128 registers (the 16 warps then share the register file), else one.
#ifndef FFCA_MAX_GROUPS
#define FFCA_MAX_GROUPS 2
#endif
template <typename T, int I, int J>
struct StreamGroups {
  static constexpr int value = (sizeof(T) == 4 && I <= 4 && J <= 3) ? FFCA_MAX_GROUPS : 1;
};

// The role of a thread in its CTA.  Warp w belongs to group (w / 4) % G with
// rank (w / (4 G)) * 4 + w % 4 in it; ranks below kConsumerWarps consume, the
// last rank produces.
struct Role {
  int group;   // pipeline group within the CTA
  int vb;      // virtual block: the partition range this group works on
  int cwarp;   // rank of the warp in its group
  int ctid;    // consumer thread index in the group (valid for consumers)
  bool consumer;
};
template <int G>
__device__ inline Role role() {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Role r;
  r.group = (w / 4) % G;
  r.cwarp = (w / (4 * G)) * 4 + w % 4;
  r.vb = (int)blockIdx.x * G + r.group;
  r.consumer = r.cwarp < kConsumerWarps;
  r.ctid = r.cwarp * 32 + lane;
  return r;
}

// A tile is up to T vector units of one frequency: I y rows of 16-byte units
// and J v rows of 8-byte units, contiguous in global memory per row.  T is
// one or two units per consumer thread (always even).  Each stage also
// carries the tile's per-frequency parameters (a ParamsA or ParamsB record),
// so a consumer starting a new frequency finds them already in shared memory.
template <typename R, int I, int J, int GG = StreamGroups<R, I, J>::value>
struct Tile {
  static constexpr int G = GG;  // pipeline groups per CTA
  static constexpr int UB = 16 * I + 8 * J;                      // bytes per unit over all rows
  static constexpr int PARAMS = ParamsA<double, I, J>::BYTES;     // room for either record
  // FFCA_TILE_UNITS_PER_THREAD units per consumer thread where three stages
  // of that size fit the budget, else one
  static constexpr int T = (((kStreamSmemBudget - (I > 4 ? 32 * 1024 : 0)) / G) /
                                    (FFCA_TILE_UNITS_PER_THREAD * kConsumers * UB + PARAMS + 16) >= 3
                                ? FFCA_TILE_UNITS_PER_THREAD
                                : 1) *
                           kConsumers;  // units per tile
  // stage layout: I y rows of YP 16-byte units (pitch skewed by one unit for
  // I > 4, whose pass-B consumers read I rows at the same unit in one
  // instruction: the skew puts them in distinct banks), J v rows of T
  // 8-byte units, the parameter record
  static constexpr int YP = T + (I > 4 ? 1 : 0);
  static constexpr int VOFF = I * YP * 16;                        // byte offset of the v rows
  static constexpr int ROFF = VOFF + J * T * 8;                   // byte offset of the record
  static constexpr int STAGE = ROFF + PARAMS;                     // bytes per stage, multiple of 16
  // I > 4: pass B's static reduction buffer (I^3 sums of 7 warps, two floats) takes ~29 KB
  static constexpr int BUDGET = kStreamSmemBudget - (I > 4 ? 32 * 1024 : 0);
  static constexpr int S_FIT = (BUDGET / G) / (STAGE + 16);
  static constexpr int S = S_FIT < 2 ? 2 : (S_FIT > FFCA_MAX_STAGES ? FFCA_MAX_STAGES : S_FIT);  // stages
  static constexpr int GROUP = S * STAGE + 2 * S * 8;             // + mbarriers
  static_assert(G * GROUP + (I > 4 ? 32 * 1024 : 0) <= 227 * 1024, "stages exceed the shared memory of a CTA");
};

// Pipelines per CTA of pass A in its EM form (k_estep<..., EM = true>):
// with P and Lambda read from the stage's record at each use (not held in
// registers), the FP32 form fits two groups of 128 registers for I <= 3,
// J <= 3; else one group.
#ifndef FFCA_EM_GROUPS
#define FFCA_EM_GROUPS 2
#endif
template <typename T, int I, int J>
struct EmGroups {
  static constexpr int value = (sizeof(T) == 4 && I <= 3 && J <= 3) ? FFCA_EM_GROUPS : 1;
};

// Pipelines per CTA of pass B: as pass A (at I = 8 one group: the
// per-thread sums of wcov_consume_big take 222 registers; a sixteen-thread
// entry split that fits two groups of 128 registers ran slower, 157.8 against
// 137 us at I = 8, J = 6, F = 513, N = 4000).
#ifndef FFCA_BIG_B_GROUPS
#define FFCA_BIG_B_GROUPS 1
#endif
template <typename T, int I, int J>
struct WcovGroups {
  static constexpr int value = I > 4 ? (sizeof(T) == 4 ? FFCA_BIG_B_GROUPS : 1) : StreamGroups<T, I, J>::value;
};

// Register cap of the streaming kernels: 128 for two groups per CTA, else
// what one group of eight warps may use.
template <typename T, int I, int J>
struct StreamRegs {
  static constexpr int value = StreamGroups<T, I, J>::value == 2 ? 128 : 255;
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
// Barrier over the consumer warps of one group (named barrier 1 + group).
__device__ inline void consumer_sync(int group) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "n"(kConsumers) : "memory");
}

// Reduction of NV per-thread values over a group's consumer warps:
// a butterfly reduce-scatter inside each warp (at level `off` every lane
// keeps half of its remaining values and receives the partner's partial
// sums of that half from lane ^ off: 31 exchanges reduce 32 values where a
// tree per value needs 5 each; lane l ends with value l of its chunk), in
// plain arithmetic (a pairwise tree of five levels), then the seven warp
// results summed in shared memory in warp order, compensated in FP32
// (double-float: TwoSum of each addition, errors carried), written as FP64.
// A segment's per-thread sums cover few frames when problems are short (the
// batched workload: ~4 units per thread), so this reduction runs about as
// often as the per-point work; a compensated butterfly (two shuffles and a
// double-float addition per exchange) made it half of pass B's instructions
// there.  Consumer thread t < NV writes value t to out[t].
// The warp partials alternate between two buffers from one segment to the
// next (parity), so one barrier per segment suffices: a thread writes the
// buffer of segment s + 2 only after the barrier of segment s + 1, which
// every thread reaches after its reads of segment s.
template <typename T, int NV, int NB = 2>
struct GroupReduce {
  static constexpr int NC = (NV + 31) / 32;  // chunks of 32 values
  static constexpr bool PAIR = sizeof(T) == 4;
  struct Smem {
    T hi[NB][kConsumerWarps][NC * 32];  // NB = 1: single buffer, two barriers per segment
  };
  // single-buffered view (the I > 4 pass B, two barriers per segment)
  __device__ static T (&one(Smem& sm))[kConsumerWarps][NC * 32] { return sm.hi[0]; }

  // add: add the values to out[] (a later flush of the same segment) instead
  // of storing them
  __device__ static void run(const T (&hi)[NV], Smem& smem, double* out, const Role& r, int parity,
                             bool add = false) {
    static_assert(NB == 2, "run() alternates two buffers");
    auto& sm = smem.hi[parity & 1];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T h[32];
#pragma unroll
      for (int v = 0; v < 32; ++v) {
        const int idx = c * 32 + v;
        h[v] = idx < NV ? hi[idx] : (T)0;
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
          const T kh = up ? h[j + off] : h[j];
          const T sh = up ? h[j] : h[j + off];
          h[j] = kh + __shfl_xor_sync(0xffffffffu, sh, off);
        }
      }
      sm[r.cwarp][c * 32 + lane] = h[0];
    }
    consumer_sync(r.group);
    for (int t = r.ctid; t < NV; t += kConsumers) {
      T h = sm[0][t];
      T l = (T)0;
#pragma unroll
      for (int w = 1; w < kConsumerWarps; ++w) {
        if constexpr (PAIR) {
          df_add(h, l, sm[w][t], (T)0);
        } else {
          h += sm[w][t];
        }
      }
      const double x = (double)h + (double)l;
      out[t] = add ? out[t] + x : x;
    }
  }
};

// Flushes of the per-thread FP32 sums that cannot be compensated in
// registers (more sums than the register file holds twice): a group reduces
// its sums into its slot every kFlushUnits units per thread of a segment,
// adding to what earlier flushes of the segment stored (FP64), so that no
// thread's plain FP32 sum runs over more than kFlushUnits units, however
// long the problem is.  Tile trips between flushes for UPT units per thread
// per trip:
constexpr int kFlushUnits = 64;
// Tile trips between the Kahan steps of the compensated sums (KSum): a
// thread's partial covers at most this many trips' units (two per trip at
// most) before it is folded into the running total.
constexpr int kFoldTiles = 4;
__host__ __device__ constexpr int flush_tiles(int upt) { return kFlushUnits / upt > 0 ? kFlushUnits / upt : 1; }

// Tiles of a CTA's unit range [u0, u1) of the flattened unit space: at most
// T units each, never crossing a problem boundary (tile = problem f, first
// unit k within the problem, n units).  The problem index is found once
// (binary search over the unit starts) and then stepped as the walk crosses
// into the neighbouring problem.  Forward walks go from u0 up, reverse walks
// from u1 down: pass A walks forward and pass B in reverse, so that each pass
// starts on the units the previous pass touched last, which are still in
// the 129 MB L2 (the two passes have the same ranges when their partitions
// agree).  Tile starts stay even (16-byte aligned v rows): ranges, problem
// starts and T are even.
struct TileIter {
  const Partition* pt;
  long long u, u0, u1;
  long long s, e;  // unit range of problem f
  int T;
  int f, k, n;
  bool seg_end, rev;
  __device__ TileIter(long long u0_, long long u1_, const Partition& pt_, int T_, bool rev_ = false)
      : pt(&pt_), u(rev_ ? u1_ : u0_), u0(u0_), u1(u1_), T(T_), rev(rev_) {
    f = u0 < u1 ? pt->problem_of(rev ? u1 - 1 : u0) : 0;
    s = pt->start(f);
    e = pt->start(f + 1);
  }
  __device__ bool next() {
    if (!rev) {
      if (u >= u1) return false;
      if (u >= e) {  // ranges are contiguous: the next problem starts at e
        ++f;
        s = e;
        e = pt->start(f + 1);
      }
      k = (int)(u - s);
      const int kend = (int)(min(e, u1) - s);
      n = min(T, kend - k);
      seg_end = (k + n == kend);
      u += n;
    } else {
      if (u <= u0) return false;
      if (u <= s) {  // the previous problem ends at s
        --f;
        e = s;
        s = pt->start(f);
      }
      const int kbeg = (int)(max(s, u0) - s);
      const int kend = (int)(u - s);
      n = min(T, kend - kbeg);
      k = kend - n;
      seg_end = (k == kbeg);
      u -= n;
    }
    return true;
  }
  // the problem the walk reaches after f, or -1 if f is its last
  __device__ int after(int p) const {
    if (!rev) return (p + 1 < pt->F && pt->start(p + 1) < u1) ? p + 1 : -1;
    return (p > 0 && pt->start(p) > u0) ? p - 1 : -1;
  }
};

template <int S>
struct Pipe {
  static constexpr int kStages = S;
  unsigned char* smem;
  uint32_t bars;  // full[s] at bars + 8 s, empty[s] at bars + 8 (S + s)
  __device__ uint32_t full(int s) const { return bars + 8 * s; }
  __device__ uint32_t empty(int s) const { return bars + 8 * (S + s); }
};

// Pass B's parameters for problem f, computed by its producer warp from pass
// A's slots (FP64, one value per lane, slot order): the new Lambda (Eq.
// Lambdaupdate, lambda_ji I sum_n t_ji / s_j / N with the slot sums of
// k_estep); lane q < J I returns entry q.  The CTA that starts problem f also
// stores the new Lambda (committed to lambda by k_psolve, after every CTA of
// this pass has read the current one) and the problem's log-likelihood of
// the state entering the iteration (Eq. L2).  The loads (FinIn) are issued
// one problem ahead and held as loaded (up to four slots), so that the
// producer does not wait for them while it issues the current problem's
// copies; their sums are formed when used (pass B 73.1 -> 71.3 us at the
// long mixture against summing at load time).  Called by all 32 lanes.
template <int I, int J>
struct FinIn {
  static constexpr int NC = (J * I + 2 + 31) / 32;  // values per lane
  static constexpr int KPF = 4;  // slots held as loaded, summed when used
  double raw[NC][KPF];  // value q = lane + 32 c < J I + 2: slots 0 .. KPF-1
  double rest[NC];      // slots KPF and up, summed at load time
  int ns;               // slots of the problem
  double x[NC];         // q < J I: current lambda entry q; q = J I: ln|det P|^2
  // value c's slot sum, slot order (the loads of the first KPF slots have
  // long landed when the sums are used, one problem later)
  __device__ double tot(int c) const {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < KPF; ++k)
      if (k < ns) t += raw[c][k];
    return ns > KPF ? t + rest[c] : t;
  }
};

template <int I, int J>
__device__ inline FinIn<I, J> finalize_load(const FastArgs& a, int f) {
  constexpr int NA = J * I;
  constexpr int NV = NA + 2;
  using FI = FinIn<I, J>;
  const int lane = threadIdx.x & 31;
  const Partition& pa = a.prev_part;
  const int ns = pa.nslots(f);
  const double* p = a.prev_buf + ((size_t)f * pa.max_slots) * NV;
  FI in;
  in.ns = ns;
#pragma unroll
  for (int c = 0; c < FI::NC; ++c) {
    const int q = lane + 32 * c;
    in.x[c] = 0.0;
    in.rest[c] = 0.0;
#pragma unroll
    for (int k = 0; k < FI::KPF; ++k) in.raw[c][k] = (q < NV && k < ns) ? __ldcg(p + (size_t)k * NV + q) : 0.0;
    if (q < NV)
      for (int k = FI::KPF; k < ns; ++k) in.rest[c] += __ldcg(p + (size_t)k * NV + q);
    if (q < NA)
      in.x[c] = __ldcg(a.lam + (size_t)f * NA + q);
    else if (q == NA)
      in.x[c] = __ldcg(a.logdet + f);
  }
  return in;
}

// Returns this lane's entries (q = lane + 32 c) of the new Lambda in out[c].
template <typename T, int I, int J>
__device__ void finalize_pass_a(const FastArgs& a, int f, const FinIn<I, J>& in, bool first,
                                T (&out)[FinIn<I, J>::NC]) {
  constexpr int NA = J * I;
  using FI = FinIn<I, J>;
  const int lane = threadIdx.x & 31;
  // the log2-sum lives at q = NA + 1: chunk (NA + 1) / 32, lane (NA + 1) % 32
  const double lg = __shfl_sync(0xffffffffu, in.tot((NA + 1) / 32), (NA + 1) % 32);
  bool bad = false;
#pragma unroll
  for (int c = 0; c < FI::NC; ++c) {
    const int q = lane + 32 * c;
    out[c] = (T)0;
    if (q < NA) {
      const double lnew = in.x[c] * ((double)I * a.part.inv_n(f)) * in.tot(c);
      bad |= !(lnew > 0.0) || !isfinite(lnew);
      out[c] = (T)lnew;
      if (first) a.lam_next[(size_t)f * NA + q] = lnew;
    } else if (q == NA && first) {
      const int n = a.part.frames(f);
      const double lf = -(double)I * n * kLnPi + (double)n * in.x[c] - in.tot(c) - 0.69314718055994530942 * lg;
      bad |= !isfinite(lf);
      a.llf[f] = lf;
    }
  }
  if (bad) raise_status(a.status, kDevNonfinite, f);
}

// Producer: one thread in pass A, the whole warp in pass B (lane 0 issues
// the copies; the warp finalises pass A's sums of each new problem).  y units
// are 16 bytes, v units 8 bytes; ranges start on even units, so every copy is
// 16-byte aligned and a multiple of 16 bytes.  Each stage also receives the
// tile's parameter record: copied from the pass-A table (pass A), or computed
// from pass A's slots (pass B).
template <typename T, int I, int J, bool PASS_B, int G = StreamGroups<T, I, J>::value>
__device__ void produce(const FastArgs& a, const Pipe<Tile<T, I, J, G>::S>& pp, long long u0, long long u1,
                        long long row, int vb, volatile int* abort) {
  using TC = Tile<T, I, J, G>;
  constexpr int kStages = TC::S;
  using PA = ParamsA<T, I, J>;
  using PB = ParamsB<T, I, J>;
  constexpr int NA = J * I;
  const char* y = static_cast<const char*>(a.y);
  const char* v = static_cast<const char*>(a.v);
  const char* tab = static_cast<const char*>(a.tabA);
  constexpr int FU = Vec<T>::FU;
  const bool leader = (threadIdx.x & 31) == 0;
  const Partition& pt = a.part;
  TileIter it(u0, u1, pt, TC::T, PASS_B);
  using FI = FinIn<I, J>;
  T lam_q[FI::NC];  // pass B: this lane's entries of the current problem's new Lambda
  FI next_in;
  if (PASS_B && u1 > u0) next_in = finalize_load<I, J>(a, it.f);
  int pf = -1;
  int t = 0;
  while (it.next()) {
    const int s = t % kStages;
    if (PASS_B && it.f != pf) {
      const FI cur = next_in;
      const int nf = it.after(it.f);
      if (nf >= 0) next_in = finalize_load<I, J>(a, nf);
      finalize_pass_a<T, I, J>(a, it.f, cur, pt.first_block(it.f) == vb, lam_q);
      pf = it.f;
    }
    int stop = 0;
    if (leader) {
      if (t >= kStages && !*abort && !mbar_wait(pp.empty(s), ((t / kStages) - 1) & 1)) {
        raise_status(a.status, kDevTimeout, it.f);
        *abort = 1;
      }
      stop = *abort;
    }
    if constexpr (PASS_B) stop = __shfl_sync(0xffffffffu, stop, 0);  // one decision for the warp
    if (stop) break;
    unsigned char* stp = pp.smem + (size_t)s * TC::STAGE;
    const uint32_t st = smem_u32(stp);
    if constexpr (PASS_B) {
      // lane q < J I stores its entry of the parameter record; the warp
      // barrier orders these stores before lane 0's arrive, which releases
      // them to the consumers together with the tile
#pragma unroll
      for (int c = 0; c < FI::NC; ++c) {
        const int q = (int)(threadIdx.x & 31) + 32 * c;
        if (q < NA) (&reinterpret_cast<PB*>(stp + TC::ROFF)->lam[0][0])[q] = lam_q[c];
      }
      __syncwarp();
      if (!leader) {
        ++t;
        continue;
      }
      mbar_expect_tx(pp.full(s), (unsigned)(it.n * TC::UB));
    } else {
      mbar_expect_tx(pp.full(s), (unsigned)(it.n * TC::UB + PA::BYTES));
      bulk_g2s(st + TC::ROFF, tab + (size_t)it.f * PA::BYTES, (unsigned)PA::BYTES, pp.full(s));
    }
    // rows of the problem's blocks (units): mic m at I Fm off + (m Fm + f) ld,
    // source j at J Fm off + (j Fm + f) ld (frames / FU)
    const long long rlen = pt.row_len(it.f, row * FU) / FU;
    const long long off = pt.frame_off(it.f) / FU;
    const long long r0 = (long long)pt.freq(it.f) * rlen + it.k;
#pragma unroll
    for (int m = 0; m < I; ++m)
      bulk_g2s(st + m * TC::YP * 16, y + ((size_t)I * pt.Fm * off + (size_t)m * pt.Fm * rlen + r0) * 16,
               (unsigned)it.n * 16, pp.full(s));
#pragma unroll
    for (int j = 0; j < J; ++j)
      bulk_g2s(st + TC::VOFF + j * TC::T * 8,
               v + ((size_t)J * pt.Fm * off + (size_t)j * pt.Fm * rlen + r0) * 8, (unsigned)it.n * 8, pp.full(s));
    ++t;
  }
  // let the copies of the last stages land before this thread leaves
  if (leader)
    for (int d = t > kStages ? t - kStages : 0; d < t; ++d) mbar_wait(pp.full(d % kStages), (d / kStages) & 1);
}

// Every group's stages and mbarriers, initialised by thread 0; returns this
// thread's group pipe.
template <int G, int S>
__device__ inline Pipe<S> setup_pipe(unsigned char* smem, int stage_bytes, int group, volatile int* aborts) {
  const size_t group_bytes = (size_t)S * stage_bytes + 2 * S * 8;
  auto pipe_of = [&](int g) {
    Pipe<S> p;
    p.smem = smem + g * group_bytes;
    p.bars = smem_u32(p.smem + (size_t)S * stage_bytes);
    return p;
  };
  if (threadIdx.x == 0) {
    for (int g = 0; g < G; ++g) {
      const Pipe<S> p = pipe_of(g);
      for (int s = 0; s < S; ++s) {
        mbar_init(p.full(s), 1);
        mbar_init(p.empty(s), kConsumerWarps);
      }
      aborts[g] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  return pipe_of(group);
}

// Consumer side of one tile: wait for it unless the CTA has given up.
template <int S>
__device__ inline bool consumer_acquire(const FastArgs& a, const Pipe<S>& pp, int t, int f, volatile int* abort) {
  if (*abort) return false;
  if (mbar_wait(pp.full(t % S), (t / S) & 1)) return true;
  raise_status(a.status, kDevTimeout, f);
  *abort = 1;
  return false;
}
template <int S>
__device__ inline void consumer_release(const Pipe<S>& pp, int t) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(pp.empty(t % S));
}

// ------------------------------------------------------------ frame lanes
// The frames of one vector unit are processed together: the two c64 frames
// as one packed pair with Blackwell's f32x2 FMA / MUL / ADD (one instruction
// for both frames), the single c128 frame as a plain double.
struct F2 {
  float2 v;
};
__device__ inline F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ inline F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ inline F2 vfma(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ inline F2 vrcp(F2 x) {  // hardware approximation + one Newton-Raphson step
  F2 r = {make_float2(0.f, 0.f)};
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.v.x) : "f"(x.v.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.v.y) : "f"(x.v.y));
  const F2 e = vfma(x * F2{make_float2(-1.f, -1.f)}, r, F2{make_float2(1.f, 1.f)});  // 1 - x r
  return vfma(r, e, r);
}
__device__ inline F2 vlog2(F2 x) { return {make_float2(__log2f(x.v.x), __log2f(x.v.y))}; }

struct D1 {
  double v;
};
__device__ inline D1 operator+(D1 a, D1 b) { return {a.v + b.v}; }
__device__ inline D1 operator*(D1 a, D1 b) { return {a.v * b.v}; }
__device__ inline D1 vfma(D1 a, D1 b, D1 c) { return {fma(a.v, b.v, c.v)}; }
__device__ inline D1 vrcp(D1 x) { return {recip(x.v)}; }
__device__ inline D1 vlog2(D1 x) { return {log2(x.v)}; }

// sum_i log2 sigma_i of one point in FP32 lanes: one hardware log2 per
// sigma.  (FP64 keeps a running product of the sigmas' binary mantissas
// over a thread's points instead, with one software logarithm per segment:
// see the pass-A consumer.)
template <typename L>
struct Log2Sum;
template <>
struct Log2Sum<F2> {
  F2 s = {make_float2(0.f, 0.f)};
  __device__ inline void add(F2 x) { s = s + vlog2(x); }
  __device__ inline F2 value() const { return s; }
};
template <>
struct Log2Sum<D1> {};  // unused: FP64 takes the running product

template <typename T>
struct Lane;
template <>
struct Lane<float> {
  using L = F2;
  __device__ static L bc(float x) { return {make_float2(x, x)}; }
  __device__ static void split(const float4& u, L& re, L& im) {
    re = {make_float2(u.x, u.z)};
    im = {make_float2(u.y, u.w)};
  }
  __device__ static L real(const float2& u) { return {u}; }
  __device__ static float2 store(L x) { return x.v; }
  // zero the lanes of frames at or beyond N (frame index n0 of lane 0)
  __device__ static L keep(L x, int n0, int N) {
    return {make_float2(n0 < N ? x.v.x : 0.f, n0 + 1 < N ? x.v.y : 0.f)};
  }
  __device__ static L pick(L fresh, L old, int n0, int N) {
    return {make_float2(n0 < N ? fresh.v.x : old.v.x, n0 + 1 < N ? fresh.v.y : old.v.y)};
  }
  __device__ static double total(L x) { return (double)x.v.x + (double)x.v.y; }
  __device__ static float hsum(L x) { return x.v.x + x.v.y; }
};
template <>
struct Lane<double> {
  using L = D1;
  __device__ static L bc(double x) { return {x}; }
  __device__ static void split(const double2& u, L& re, L& im) {
    re = {u.x};
    im = {u.y};
  }
  __device__ static L real(double u) { return {u}; }
  __device__ static double store(L x) { return x.v; }
  __device__ static L keep(L x, int n0, int N) { return {n0 < N ? x.v : 0.0}; }
  __device__ static L pick(L fresh, L old, int n0, int N) { return {n0 < N ? fresh.v : old.v}; }
  __device__ static double hsum(L x) { return x.v; }
};

// -------------------------------------------------------------- shuffles of frame lanes
__device__ inline F2 shfl_xor_l(F2 x, int off) {
  return {make_float2(__shfl_xor_sync(0xffffffffu, x.v.x, off), __shfl_xor_sync(0xffffffffu, x.v.y, off))};
}
__device__ inline D1 shfl_xor_l(D1 x, int off) { return {__shfl_xor_sync(0xffffffffu, x.v, off)}; }
__device__ inline F2 shfl_l(F2 x, int src) {
  return {make_float2(__shfl_sync(0xffffffffu, x.v.x, src), __shfl_sync(0xffffffffu, x.v.y, src))};
}
__device__ inline D1 shfl_l(D1 x, int src) { return {__shfl_sync(0xffffffffu, x.v, src)}; }
__device__ inline float lane_of(F2 x, int fr) { return fr == 0 ? x.v.x : x.v.y; }
__device__ inline double lane_of(D1 x, int) { return x.v; }

// -------------------------------------------------------------- pass A, EM form, I > 4
// The normal EM update of P (Sec. 4.6) needs, beyond pass A's sums, the
// J I (I - 1) sums u_j z_a conj(z_b) (a < b; z_a = r_a y~_a, u_j = v_j / s_j,
// as in k_estep) per point: 336 at I = 8, J = 6, more than one thread holds.
// So each unit is shared by I threads, as in pass B's I > 4 form: thread e
// of a unit forms y~_e = sum_m conj(P_me) y_m, sigma_e, r_e and t_je
// (Eq. updatev's terms of i = e); the unit's threads add t_je over e by a
// butterfly (s_j in every lane); thread e < J writes v_e^new; each thread
// keeps the Lambda sums of its column e (sum_n t_je / s_j), the L2 terms of
// i = e, and the EM sums of the pairs p = SL e .. SL e + SL - 1 (row order
// over a < b; thread I - 1 none), taking z_a and z_b of a pair from their
// lanes by shuffles.  The slot holds the I <= 4 form's layout: the Lambda
// sums, the two L2 sums, then (re, im) per j and pair.
template <int I, int J>
struct EmBig {
  static constexpr int PAIRS = I * (I - 1) / 2;
  static constexpr int SL = (PAIRS + I - 1) / I;      // pair slots per thread (4 at I = 8)
  static constexpr int NVT = J + 2 + 2 * J * SL;      // values per thread
  static constexpr int NA = J * I;
  static constexpr int NV = NA + 2 + 2 * J * PAIRS;   // values per slot
  // row and column of pair p (row order over a < b)
  __device__ static void decode(int p, int& ra, int& cb) {
    ra = 0;
    int q = p;
    while (q >= I - 1 - ra) {
      q -= I - 1 - ra;
      ++ra;
    }
    cb = ra + 1 + q;
  }
  // slot index of thread e's value v, or -1 (an unused pair slot; the L2
  // parts of the threads e > 0, which the reduction leaves in thread 0)
  __device__ static int out_index(int e, int v) {
    if (v < J) return v * I + e;
    if (v < J + 2) return e == 0 ? NA + (v - J) : -1;
    const int w = v - J - 2, k = w / (2 * J), j = (w % (2 * J)) / 2, comp = w % 2;
    const int p = SL * e + k;
    return p < PAIRS ? NA + 2 + 2 * (j * PAIRS + p) + comp : -1;
  }
};

template <typename T, int I, int J, typename Red, int S, int G>
__device__ void estep_consume_big_em(const FastArgs& a, const Pipe<S>& pp, long long u0, long long u1,
                                     const Role& rl, volatile int* abort, typename Red::Smem& red) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using LN = Lane<T>;
  using L = typename LN::L;
  using TC = Tile<T, I, J, G>;
  using PA = ParamsA<T, I, J>;
  using EB = EmBig<I, J>;
  using T2 = std::conditional_t<sizeof(T) == 4, float2, double2>;
  constexpr int FU = Vec<T>::FU;
  constexpr int SL = EB::SL, NVT = EB::NVT;
  constexpr int IG = kConsumers / I;  // units in flight per group
  static_assert(kConsumers % I == 0 && 32 % I == 0 && J <= I, "I must divide the consumer count and the warp");
  const Partition& pt = a.part;
  const int tid = rl.ctid, lane = threadIdx.x & 31;
  const int e = tid % I, ul = tid / I;
  const int gl = lane & ~(I - 1);  // first lane of this unit's I threads
  int sa[SL], sb[SL];
#pragma unroll
  for (int k = 0; k < SL; ++k) {
    const int p = SL * e + k;
    if (p < EB::PAIRS) EB::decode(p, sa[k], sb[k]);
    else { sa[k] = 0; sb[k] = 1; }  // thread I - 1: unused slots
  }
  auto fma2 = [](T w, T xr, T xi, T2 acc) -> T2 {
    if constexpr (sizeof(T) == 4) return __ffma2_rn(make_float2(w, w), make_float2(xr, xi), acc);
    else return make_double2(fma(w, xr, acc.x), fma(w, xi, acc.y));
  };
  VV* __restrict__ vg = reinterpret_cast<VV*>(a.v);
  const long long row = a.ld / FU;
  T pre[I], pim[I], lame[J];  // column e of P and lambda_je of the segment's problem
  T lacc[J], qacc, gacc;      // Lambda sums of column e, L2 parts of i = e
  T2 eacc[SL][J];             // (re, im) of u_j z_a conj(z_b) per pair slot
  TileIter it(u0, u1, pt, TC::T);
  bool seg_new = true;
  int ntile = 0;         // tile trips since the segment's start or last flush
  bool flushed = false;  // the segment has flushed into its slot
  int Np = 0;
  long long rlen = 0;
  VV* __restrict__ vrow = vg;
  for (int t = 0; it.next(); ++t) {
    const int f = it.f;
    if (seg_new) {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        lacc[j] = (T)0;
#pragma unroll
        for (int k = 0; k < SL; ++k) eacc[k][j] = T2{0, 0};
      }
      qacc = (T)0;
      gacc = (T)0;
      Np = pt.frames(f);
      rlen = pt.row_len(f, row * FU) / FU;
      vrow = vg + (size_t)J * pt.Fm * (pt.frame_off(f) / FU) + (size_t)pt.freq(f) * rlen;
    }
    if (consumer_acquire(a, pp, t, f, abort)) {
      const unsigned char* st = pp.smem + (size_t)(t % S) * TC::STAGE;
      if (seg_new) {
        const PA& sp = *reinterpret_cast<const PA*>(st + TC::ROFF);
#pragma unroll
        for (int m = 0; m < I; ++m) {
          pre[m] = sp.pre(m, e);
          pim[m] = sp.pim(m, e);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) lame[j] = sp.lam(j, e);
      }
      const VY* ys = reinterpret_cast<const VY*>(st);
      const VV* vs = reinterpret_cast<const VV*>(st + TC::VOFF);
      // every lane runs the same trips (the shuffles need the whole warp);
      // units beyond the tile get neutral data and add nothing
#pragma unroll 1
      for (int qb = 0; qb < it.n; qb += IG) {
        const int q = qb + ul;  // < T: it.n <= T and T is a multiple of IG
        const int k = it.k + q;
        const int n0 = k * FU;
        const bool unit_ok = q < it.n && n0 < Np;
        const bool full = n0 + FU <= Np;
        // y~_e = sum_m conj(P_me) y_m: re = Pr yr + Pi yi, im = Pr yi - Pi yr
        L tr = LN::bc(0), ti = LN::bc(0);
#pragma unroll
        for (int m = 0; m < I; ++m) {
          L yr = LN::bc(0), yi = LN::bc(0);
          if (unit_ok) LN::split(ys[m * TC::YP + q], yr, yi);
          const L pr = LN::bc(pre[m]), pi = LN::bc(pim[m]);
          tr = vfma(pr, yr, vfma(pi, yi, tr));
          ti = vfma(pr, yi, vfma(pi * LN::bc(-1), yr, ti));
        }
        L vv[J];
#pragma unroll
        for (int j = 0; j < J; ++j) vv[j] = unit_ok ? LN::real(vs[j * TC::T + q]) : LN::bc(1);
        L sg = vv[0] * LN::bc(lame[0]);
#pragma unroll
        for (int j = 1; j < J; ++j) sg = vfma(vv[j], LN::bc(lame[j]), sg);
        const L r = vrcp(sg);
        const L e2 = vfma(tr, tr, ti * ti);
        const L w = r * vfma(r, e2, LN::bc(-1));
        L tj[J], sj[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          tj[j] = vfma(vv[j] * LN::bc(lame[j]), w, LN::bc(1));
          sj[j] = tj[j];
        }
#pragma unroll
        for (int off = 1; off < I; off <<= 1)  // s_j = sum over the unit's I threads
#pragma unroll
          for (int j = 0; j < J; ++j) sj[j] = sj[j] + shfl_xor_l(sj[j], off);
        L rs[J];
#pragma unroll
        for (int j = 0; j < J; ++j) rs[j] = vrcp(sj[j]);
        const L zr = r * tr, zi = r * ti;
        L zar[SL], zai[SL], zbr[SL], zbi[SL];
#pragma unroll
        for (int kk = 0; kk < SL; ++kk) {
          zar[kk] = shfl_l(zr, gl | sa[kk]);
          zai[kk] = shfl_l(zi, gl | sa[kk]);
          zbr[kk] = shfl_l(zr, gl | sb[kk]);
          zbi[kk] = shfl_l(zi, gl | sb[kk]);
        }
        if (!unit_ok) continue;  // after the shuffles: nothing below involves other lanes
        if (e < J) {  // v^new of source e (the padding frames of a ragged unit keep their values)
          L ve = vv[0], se = sj[0];
#pragma unroll
          for (int j = 1; j < J; ++j)
            if (j == e) {
              ve = vv[j];
              se = sj[j];
            }
          const L vn = ve * se * LN::bc((T)(1.0 / I));
          vrow[(size_t)e * pt.Fm * rlen + k] = LN::store(full ? vn : LN::pick(vn, ve, n0, Np));
        }
        L uj[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          uj[j] = vv[j] * rs[j];
          L x = tj[j] * rs[j];
          if (!full) {  // padding frames may hold anything: select, do not multiply
            x = LN::keep(x, n0, Np);
            uj[j] = LN::keep(uj[j], n0, Np);
          }
          lacc[j] += LN::hsum(x);
        }
        {
          L qd = e2 * r, lg = vlog2(sg);
          if (!full) {
            qd = LN::keep(qd, n0, Np);
            lg = LN::keep(lg, n0, Np);
          }
          qacc += LN::hsum(qd);
          gacc += LN::hsum(lg);
        }
#pragma unroll
        for (int kk = 0; kk < SL; ++kk) {
          const L pr = vfma(zar[kk], zbr[kk], zai[kk] * zbi[kk]);                 // re(z_a conj(z_b))
          const L pi = vfma(zai[kk], zbr[kk], (zar[kk] * zbi[kk]) * LN::bc(-1));  // im(z_a conj(z_b))
#pragma unroll
          for (int fr = 0; fr < FU; ++fr) {
            if (!full && n0 + fr >= Np) continue;  // a padding frame: its values may be anything
#pragma unroll
            for (int j = 0; j < J; ++j)
              eacc[kk][j] = fma2(lane_of(uj[j], fr), lane_of(pr, fr), lane_of(pi, fr), eacc[kk][j]);
          }
        }
      }
    }
    seg_new = false;
    consumer_release(pp, t);

    // FP32: the plain sums are flushed into the slot every 2 kFlushUnits
    // units per thread, as pass B's I > 4 form
    const bool flush = sizeof(T) == 4 && !it.seg_end && ++ntile == 2 * flush_tiles(TC::T / IG);
    if (it.seg_end || flush) {
      const int slot = rl.vb - pt.first_block(f);
      double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * EB::NV;
      T h[NVT];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        h[j] = lacc[j];
#pragma unroll
        for (int kk = 0; kk < SL; ++kk) {
          h[J + 2 + 2 * (kk * J + j)] = eacc[kk][j].x;
          h[J + 2 + 2 * (kk * J + j) + 1] = eacc[kk][j].y;
        }
      }
      h[J] = qacc;
      h[J + 1] = gacc;
#pragma unroll
      for (int off = 1; off < I; off <<= 1) {  // the L2 parts over the unit's threads
        h[J] += __shfl_xor_sync(0xffffffffu, h[J], off);
        h[J + 1] += __shfl_xor_sync(0xffffffffu, h[J + 1], off);
      }
#pragma unroll
      for (int off = I; off < 32; off <<= 1)  // the lanes with the same e
#pragma unroll
        for (int v = 0; v < NVT; ++v) h[v] += __shfl_xor_sync(0xffffffffu, h[v], off);
      if (lane < I) {
#pragma unroll
        for (int v = 0; v < NVT; ++v) Red::one(red)[rl.cwarp][lane * NVT + v] = h[v];
      }
      consumer_sync(rl.group);
      for (int x = tid; x < I * NVT; x += kConsumers) {
        const int o = EB::out_index(x / NVT, x % NVT);
        if (o < 0) continue;
        T sh = Red::one(red)[0][x];
        T sl = (T)0;
#pragma unroll
        for (int w2 = 1; w2 < kConsumerWarps; ++w2) {
          if constexpr (sizeof(T) == 4) df_add(sh, sl, Red::one(red)[w2][x], (T)0);
          else sh += Red::one(red)[w2][x];
        }
        const double xv = (double)sh + (double)sl;
        out[o] = flushed ? out[o] + xv : xv;
      }
      consumer_sync(rl.group);
      ntile = 0;
      if (flush) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          lacc[j] = (T)0;
#pragma unroll
          for (int kk = 0; kk < SL; ++kk) eacc[kk][j] = T2{0, 0};
        }
        qacc = (T)0;
        gacc = (T)0;
        flushed = true;
      } else {
        flushed = false;
        seg_new = true;
      }
    }
  }
}

// Pass A in its EM form for I > 4: the producer of k_estep, the consumers of
// estep_consume_big_em; one pipeline group per CTA.
template <typename T, int I, int J>
__global__ void __maxnreg__(255) k_estep_em_big(FastArgs a) {
  static_assert(I > 4 && EmGroups<T, I, J>::value == 1, "the I > 4 EM form runs one group per CTA");
  constexpr int G = 1;
  using TC = Tile<T, I, J, G>;
  constexpr int FU = Vec<T>::FU;
  using Red = GroupReduce<T, I * EmBig<I, J>::NVT, 1>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ typename Red::Smem red_all[G];
  __shared__ int aborts[G];
  const Role rl = role<G>();
  volatile int* abort = &aborts[rl.group];
  const Partition pt = a.part;
  const long long u0 = pt.block_start(rl.vb);
  const long long u1 = pt.block_start(rl.vb + 1);
  const long long row = a.ld / FU;
  const Pipe<TC::S> pp = setup_pipe<G, TC::S>(smem, TC::STAGE, rl.group, aborts);
  if (!rl.consumer) {
    if ((threadIdx.x & 31) == 0 && a.fault != kFaultPassANoCopies)
      produce<T, I, J, false, G>(a, pp, u0, u1, row, rl.vb, abort);
    return;
  }
  estep_consume_big_em<T, I, J, Red, TC::S, G>(a, pp, u0, u1, rl, abort, red_all[rl.group]);
}

// -------------------------------------------------------------- pass A
// Per frame, with r_i = 1/sigma_i and a_ji = v_j lambda_ji, the posterior
// power is q_ji = |mu~_ji|^2 + phi~_ji = a_ji t_ji with
// t_ji = 1 + a_ji w_i, w_i = r_i (r_i |y~_i|^2 - 1) (Eqs. mutilde0,
// Phitilde0).  Hence v_j^new = (1/I) sum_i q_ji / lambda_ji = v_j s_j / I with
// s_j = sum_i t_ji (Eq. updatev), and the Lambda numerator
// sum_n q_ji / v_j^new = I lambda_ji sum_n t_ji / s_j (Eq. Lambdaupdate): the
// kernel accumulates sum_n t_ji / s_j and k_afinal scales it.  The
// log-likelihood terms are sum_n sum_i (ln sigma_i + |y~_i|^2 r_i) (Eq. L2),
// accumulated as the quadratic part and the base-2 log part.
//
// EM (the normal EM update of P, Sec. 4.6) adds the sums its M-step for P
// needs beyond these: with z_a = r_a y~_a and u_j = v_j / s_j, the
// off-diagonal entries of T_j = sum_n (mu~_j mu~_j^H + diag phi~_j) / v_j^new
// are T_j[a][b] = I lambda_ja lambda_jb sum_n u_j z_a conj(z_b) (mu~_ja =
// a_ja r_a y~_a, v_j^new = v_j s_j / I), so the kernel sums
// u_j z_a conj(z_b) for every j and a < b (re, im); the diagonal of T_j is
// sum_n q_ja / v_j^new = N lambda_ja^new, which the Lambda sums give.  The
// larger per-point state runs one pipeline group per CTA.
template <typename T, int I, int J, bool UPDATE, bool EM = false>
__global__ void __maxnreg__((EM ? (EmGroups<T, I, J>::value == 2 ? 128 : 255) : StreamRegs<T, I, J>::value))
    k_estep(FastArgs a) {
  static_assert(!EM || (UPDATE && I <= 4), "the EM sums are laid out for I <= 4");
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using LN = Lane<T>;
  using L = typename LN::L;
  constexpr int G = EM ? EmGroups<T, I, J>::value : StreamGroups<T, I, J>::value;
  using TC = Tile<T, I, J, G>;
  constexpr int FU = Vec<T>::FU;
  constexpr int NA = UPDATE ? J * I : 0;  // sum_n t_ji / s_j
  constexpr int NPAIR = I * (I - 1) / 2;  // EM: entries a < b of T_j
  constexpr int NE = EM ? 2 * J * NPAIR : 0;
  constexpr int NV = NA + 2 + NE;         // then the quadratic and log2 parts of L2, then the EM sums
  using Red = GroupReduce<T, NV>;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ typename Red::Smem red_all[G];
  __shared__ int aborts[G];
  using PA = ParamsA<T, I, J>;

  const Role rl = role<G>();
  volatile int* abort = &aborts[rl.group];
  typename Red::Smem& red = red_all[rl.group];
  const Partition pt = a.part;
  const long long u0 = pt.block_start(rl.vb);
  const long long u1 = pt.block_start(rl.vb + 1);
  const long long row = a.ld / FU;  // vector units per (mic or source, f) row
  const Pipe<TC::S> pp = setup_pipe<G, TC::S>(smem, TC::STAGE, rl.group, aborts);

  if (!rl.consumer) {
    // an injected fault: no copies, the consumers' waits run out
    if ((threadIdx.x & 31) == 0 && a.fault != kFaultPassANoCopies)
      produce<T, I, J, false, G>(a, pp, u0, u1, row, rl.vb, abort);
    return;
  }

  VV* __restrict__ vg = reinterpret_cast<VV*>(a.v);
  const int tid = rl.ctid;
  // I <= 4: P and Lambda in registers for the segment; I > 4 (BIG): read
  // from the stage's parameter record at each use (I^2 complex values would
  // not fit the register file)
  // (EM: as well, which frees their registers for the EM sums)
  constexpr bool BIG = I > 4;
  constexpr bool PSMEM = BIG || EM;  // P and Lambda read from the stage's record
  constexpr int RI = PSMEM ? 1 : I, RJ = PSMEM ? 1 : J;
  L pre_r[RI][RI], pim_r[RI][RI], lam_r[RJ][RI];
  const PA* spc = nullptr;
  // (re, im) of P_mi as frame-lane operands
  auto PP = [&](int m, int i, L& pr, L& pi) {
    if constexpr (PSMEM) {
      pr = LN::bc(spc->pre(m, i));
      pi = LN::bc(spc->pim(m, i));
    } else {
      pr = pre_r[m][i];
      pi = pim_r[m][i];
    }
  };
  auto LAM = [&](int j, int i) -> L {
    if constexpr (PSMEM) return LN::bc(spc->lam(j, i)); else return lam_r[j][i];
  };
  // FP32: Kahan-compensated sums (KSum, folded once per tile trip); with
  // more than 32 sums one plain float per value instead (both frames of a
  // unit go into it), which keeps them in registers.  FP64: plain sums.
  constexpr bool kNarrow = sizeof(T) == 4 && NV > 32;
  constexpr bool kComp = sizeof(T) == 4 && !kNarrow;
  using A = std::conditional_t<kNarrow, float, std::conditional_t<kComp, KSum, L>>;
  A acc[NV];
  auto ACC = [&](int q, L x) {
    if constexpr (kNarrow) {
      acc[q] += x.v.x + x.v.y;
    } else if constexpr (kComp) {
      acc[q].add(x.v.x);
      acc[q].add(x.v.y);
    } else {
      acc[q] = acc[q] + x;
    }
  };
  auto ACCF = [&](int q, L x, L y) {  // sum of x y over the unit's frames
    if constexpr (kNarrow) {
      acc[q] = fmaf(x.v.y, y.v.y, fmaf(x.v.x, y.v.x, acc[q]));
    } else if constexpr (kComp) {
      acc[q].p = fmaf(x.v.y, y.v.y, fmaf(x.v.x, y.v.x, acc[q].p));
    } else {
      acc[q] = vfma(x, y, acc[q]);
    }
  };

  // FP64: sum_n log2 of the product of the sigmas over the thread's points
  // of the segment, as one running product of binary mantissas (renormalised
  // after every point, so it stays in [1/2, 1)) and a sum of exponents; its
  // logarithm is taken once, when the segment's sums are reduced
  double lg_m = 1.0;
  int lg_e = 0;
  TileIter it(u0, u1, pt, TC::T);
  bool seg_new = true;
  int nseg = 0;           // reductions so far (reduction buffer parity)
  int ntile = 0;          // tile trips since the segment's start or last flush
  int nfold = 0;          // tile trips since the last Kahan step
  bool flushed = false;   // the segment has flushed into its slot
  int Np = 0;               // the segment's problem: frames,
  long long rlen = 0;       // units per row of its block,
  VV* __restrict__ vrow = vg;  // and its v row 0 (looked up once per segment)
  for (int t = 0; it.next(); ++t) {
    const int f = it.f;
    if (seg_new) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if constexpr (kNarrow) acc[q] = 0.f;
        else if constexpr (kComp) acc[q].zero();
        else acc[q] = LN::bc(0);
      }
      Np = pt.frames(f);
      rlen = pt.row_len(f, row * FU) / FU;
      vrow = vg + (size_t)J * pt.Fm * (pt.frame_off(f) / FU) + (size_t)pt.freq(f) * rlen;
    }
    if (consumer_acquire(a, pp, t, f, abort)) {
      const unsigned char* st = pp.smem + (size_t)(t % TC::S) * TC::STAGE;
      spc = reinterpret_cast<const PA*>(st + TC::ROFF);  // every stage carries the record
      if constexpr (!PSMEM) {
        if (seg_new) {  // this frequency's P and Lambda arrived with the tile
#pragma unroll
          for (int r = 0; r < I; ++r)
#pragma unroll
            for (int c = 0; c < I; ++c) {
              pre_r[r][c] = LN::bc(spc->pre(r, c));
              pim_r[r][c] = LN::bc(spc->pim(r, c));
            }
#pragma unroll
          for (int j = 0; j < J; ++j)
#pragma unroll
            for (int i = 0; i < I; ++i) lam_r[j][i] = LN::bc(spc->lam(j, i));
        }
      }
      const VY* ys = reinterpret_cast<const VY*>(st);
      const VV* vs = reinterpret_cast<const VV*>(st + TC::VOFF);
#pragma unroll 1
      for (int q = tid; q < it.n; q += kConsumers) {
        const int k = it.k + q;
        const int n0 = k * FU;
        if (n0 >= Np) continue;  // a unit of padding frames only
        L yre[I], yim[I], nyre[I], vv[J];
#pragma unroll
        for (int m = 0; m < I; ++m) {
          LN::split(ys[m * TC::YP + q], yre[m], yim[m]);
          nyre[m] = yre[m] * LN::bc(-1);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) vv[j] = LN::real(vs[j * TC::T + q]);
        const bool full = n0 + FU <= Np;
        L r[I], e2[I];
        L ztr[EM ? I : 1], zti[EM ? I : 1];  // EM: z_i = r_i y~_i
        L quad = LN::bc(0);
        Log2Sum<L> lgs;
#pragma unroll
        for (int i = 0; i < I; ++i) {
          // y~_i = sum_m conj(P_mi) y_m: re = Pr yr + Pi yi, im = Pr yi - Pi yr
          L pr, pi;
          PP(0, i, pr, pi);
          L tr = pr * yre[0], ti = pr * yim[0];
          tr = vfma(pi, yim[0], tr);
          ti = vfma(pi, nyre[0], ti);
#pragma unroll
          for (int m = 1; m < I; ++m) {
            PP(m, i, pr, pi);
            tr = vfma(pr, yre[m], tr);
            tr = vfma(pi, yim[m], tr);
            ti = vfma(pr, yim[m], ti);
            ti = vfma(pi, nyre[m], ti);
          }
          L sg = vv[0] * LAM(0, i);
#pragma unroll
          for (int j = 1; j < J; ++j) sg = vfma(vv[j], LAM(j, i), sg);
          r[i] = vrcp(sg);
          e2[i] = vfma(tr, tr, ti * ti);
          quad = vfma(e2[i], r[i], quad);
          if constexpr (sizeof(T) == 8) {
            int ke;
            lg_m *= frexp(LN::hsum(sg), &ke);
            lg_e += ke;
          } else {
            lgs.add(sg);
          }
          if constexpr (EM) {
            ztr[i] = r[i] * tr;
            zti[i] = r[i] * ti;
          }
        }
        if constexpr (sizeof(T) == 8) {  // one frame per unit: always full
          int ke;
          lg_m = frexp(lg_m, &ke);
          lg_e += ke;
          ACC(NA, quad);
        } else {
          const L lg = lgs.value();
          if (full) {
            ACC(NA, quad);
            ACC(NA + 1, lg);
          } else {
            ACC(NA, LN::keep(quad, n0, Np));
            ACC(NA + 1, LN::keep(lg, n0, Np));
          }
        }
        if constexpr (UPDATE) {
          L w[I];
#pragma unroll
          for (int i = 0; i < I; ++i) w[i] = r[i] * vfma(r[i], e2[i], LN::bc(-1));
          L uj[EM ? J : 1];  // EM: u_j = v_j / s_j
#pragma unroll
          for (int j = 0; j < J; ++j) {
            L tj[I];
            L sj = LN::bc(0);
#pragma unroll
            for (int i = 0; i < I; ++i) {
              tj[i] = vfma(vv[j] * LAM(j, i), w[i], LN::bc(1));
              sj = sj + tj[i];
            }
            const L rs = vrcp(sj);
            if constexpr (EM) uj[j] = vv[j] * rs;
            const L vn = vv[j] * sj * LN::bc((T)(1.0 / I));
            if (full) {
#pragma unroll
              for (int i = 0; i < I; ++i) ACCF(j * I + i, tj[i], rs);
              vrow[(size_t)j * pt.Fm * rlen + k] = LN::store(vn);
            } else {
#pragma unroll
              for (int i = 0; i < I; ++i) ACC(j * I + i, LN::keep(tj[i] * rs, n0, Np));
              vrow[(size_t)j * pt.Fm * rlen + k] = LN::store(LN::pick(vn, vv[j], n0, Np));
            }
          }
          if constexpr (EM) {
            // z_a conj(z_b) for a < b in row order, then u_j times it for every j
            int pq = 0;
#pragma unroll
            for (int aa = 0; aa < I; ++aa)
#pragma unroll
              for (int bb = aa + 1; bb < I; ++bb, ++pq) {
                const L zre = vfma(ztr[aa], ztr[bb], zti[aa] * zti[bb]);
                const L zim = vfma(zti[aa], ztr[bb], (ztr[aa] * zti[bb]) * LN::bc(-1));
#pragma unroll
                for (int j = 0; j < J; ++j) {
                  const int q0 = NA + 2 + 2 * (j * NPAIR + pq);
                  if (full) {
                    ACCF(q0, uj[j], zre);
                    ACCF(q0 + 1, uj[j], zim);
                  } else {  // padding frames may hold anything: select, do not multiply
                    ACC(q0, LN::keep(uj[j] * zre, n0, Np));
                    ACC(q0 + 1, LN::keep(uj[j] * zim, n0, Np));
                  }
                }
              }
          }
        }
      }
      if constexpr (kComp) {  // one Kahan step every kFoldTiles tile trips
        if (++nfold == kFoldTiles) {
          nfold = 0;
#pragma unroll
          for (int q = 0; q < NV; ++q) acc[q].fold();
        }
      }
    }

    seg_new = false;
    consumer_release(pp, t);

    // plain FP32 sums (kNarrow) are flushed into the slot every kFlushUnits
    // units per thread; the same tiles reach every consumer of the group
    const bool flush = kNarrow && !it.seg_end && ++ntile == flush_tiles(TC::T / kConsumers);
    if (it.seg_end || flush) {
      const int slot = rl.vb - pt.first_block(f);
      double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * NV;
      if constexpr (kNarrow) {
        Red::run(acc, red, out, rl, nseg, flushed);
      } else if constexpr (kComp) {
        float hi[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) hi[q] = acc[q].value();
        Red::run(hi, red, out, rl, nseg);
      } else {
        double hi[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) hi[q] = acc[q].v;
        hi[NA + 1] += log2(lg_m) + (double)lg_e;
        lg_m = 1.0;
        lg_e = 0;
        Red::run(hi, red, out, rl, nseg);
      }
      ++nseg;  // the next reduction goes through the other buffer
      ntile = 0;
      if (flush) {
        if constexpr (kNarrow) {
#pragma unroll
          for (int q = 0; q < NV; ++q) acc[q] = 0.f;
        }
        flushed = true;
      } else {
        flushed = false;
        seg_new = true;
      }
    }
  }
}

// Pass B consumers for I > 4: the I^3 sums per point do not fit one thread's
// registers, so each unit is shared by I = 8 threads that split the entries
// of y y^H, not the weights: thread e of a unit accumulates the diagonal
// entry |y_e|^2 and the off-diagonal entries y_r conj(y_c) of the pairs
// p = 4e .. 4e+3 (row order over r < c; thread 7 only its diagonal), each
// against all I weights 1/sigma_i.  Thread e forms sigma_e and 1/sigma_e for
// the unit's frames and the I threads exchange them by shuffles, so every
// weight is computed once.  An off-diagonal entry is accumulated as one
// (re, im) pair per weight with the packed f32x2 FMA.  At a segment's end
// the lanes with the same e (equal mod 8) are summed by shuffles, then the
// warps through shared memory, in double-float; the values go out in the
// packed Hermitian order of V_i (diagonal, then (re, im) above it).
template <int I>
struct BigEntries {
  static constexpr int PAIRS = I * (I - 1) / 2;         // off-diagonal entries
  static constexpr int SLOTS = (PAIRS + I - 1) / I;     // per thread (4 at I = 8)
  static constexpr int NVT = I + 2 * I * SLOTS;         // values per thread: diagonal + slots
  static_assert(I == 8, "the entry split is laid out for I = 8");
  // packed-order index of pair p (row order over r < c) and its (r, c)
  __device__ static void decode(int p, int& r, int& c) {
    r = 0;
    int q = p;
    while (q >= I - 1 - r) {
      q -= I - 1 - r;
      ++r;
    }
    c = r + 1 + q;
  }
  // reduction index of thread e's value v (threads below I - 1 keep all NVT
  // values, thread I - 1 only its I diagonal sums): I^3 indices in all
  __device__ static int red_index(int e, int v) { return e * NVT + v; }
  // output index (weight i, packed entry m) of reduction index x
  __device__ static int out_index(int x) {
    const int e = x / NVT, v = x % NVT;
    if (v < I) return v * I * I + e;  // diagonal |y_e|^2 against weight v
    const int k = (v - I) / (2 * I), i = ((v - I) % (2 * I)) / 2, comp = (v - I) % 2;
    return i * I * I + I + 2 * (SLOTS * e + k) + comp;
  }
};

template <typename T, int I, int J, typename Red, int S, int G>
__device__ void wcov_consume_big(const FastArgs& a, const Pipe<S>& pp, long long u0, long long u1, const Role& rl,
                                 volatile int* abort, typename Red::Smem& red) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using LN = Lane<T>;
  using L = typename LN::L;
  using TC = Tile<T, I, J, G>;
  using PB = ParamsB<T, I, J>;
  using BE = BigEntries<I>;
  using T2 = std::conditional_t<sizeof(T) == 4, float2, double2>;
  constexpr int FU = Vec<T>::FU;
  constexpr int SL = BE::SLOTS;
  constexpr int IG = kConsumers / I;  // units in flight per group
  static_assert(kConsumers % I == 0 && 32 % I == 0, "I must divide the consumer count and the warp");
  const Partition& pt = a.part;
  const int tid = rl.ctid, lane = threadIdx.x & 31;
  const int e = tid % I, ul = tid / I;
  const int gl = lane & ~(I - 1);  // first lane of this unit's I threads
  int sr[SL], sc[SL];
#pragma unroll
  for (int k = 0; k < SL; ++k) {
    const int p = SL * e + k;
    if (p < BE::PAIRS) BE::decode(p, sr[k], sc[k]);
    else { sr[k] = 0; sc[k] = 1; }  // thread I - 1: unused slots
  }
  L lame[J];
  L accd[I];        // diagonal |y_e|^2 / sigma_i, per frame lane
  T2 acco[SL][I];   // off-diagonal (re, im) / sigma_i
  auto fma2 = [](T w, T xr, T xi, T2 acc) -> T2 {
    if constexpr (sizeof(T) == 4) return __ffma2_rn(make_float2(w, w), make_float2(xr, xi), acc);
    else return make_double2(fma(w, xr, acc.x), fma(w, xi, acc.y));
  };
  TileIter it(u0, u1, pt, TC::T, true);
  bool seg_new = true;
  int ntile = 0;         // tile trips since the segment's start or last flush
  bool flushed = false;  // the segment has flushed into its slot
  int Np = 0;  // frames of the segment's problem (looked up once per segment)
  for (int t = 0; it.next(); ++t) {
    const int f = it.f;
    if (seg_new) {
#pragma unroll
      for (int i = 0; i < I; ++i) {
        accd[i] = LN::bc(0);
#pragma unroll
        for (int k = 0; k < SL; ++k) acco[k][i] = T2{0, 0};
      }
      Np = pt.frames(f);
    }
    if (consumer_acquire(a, pp, t, f, abort)) {
      const unsigned char* st = pp.smem + (size_t)(t % S) * TC::STAGE;
      if (seg_new) {
        const PB& sp = *reinterpret_cast<const PB*>(st + TC::ROFF);
#pragma unroll
        for (int j = 0; j < J; ++j) lame[j] = LN::bc(sp.lam[j][e]);
      }
      const VY* ys = reinterpret_cast<const VY*>(st);
      const VV* vs = reinterpret_cast<const VV*>(st + TC::VOFF);
      // every lane runs the same trips (the shuffles need the whole warp);
      // units beyond the tile or frames beyond N get zero weight and data
#pragma unroll 1
      for (int qb = 0; qb < it.n; qb += IG) {
        const int q = qb + ul;  // < T: it.n <= T and T is a multiple of IG
        const int n0 = (it.k + q) * FU;
        const bool unit_ok = q < it.n && n0 < Np;
        L sg = LN::real(vs[q]) * lame[0];
#pragma unroll
        for (int j = 1; j < J; ++j) sg = vfma(LN::real(vs[j * TC::T + q]), lame[j], sg);
        L w = vrcp(sg);
        w = unit_ok ? LN::keep(w, n0, Np) : LN::bc(0);
        L wi[I];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int i = 0; i < I; ++i)
            wi[i] = {make_float2(__shfl_sync(0xffffffffu, w.v.x, gl | i), __shfl_sync(0xffffffffu, w.v.y, gl | i))};
        } else {
#pragma unroll
          for (int i = 0; i < I; ++i) wi[i] = {__shfl_sync(0xffffffffu, w.v, gl | i)};
        }
        if (!unit_ok) continue;  // after the shuffles: nothing below involves other lanes
        const bool ragged = n0 + FU > Np;
        // the diagonal entry |y_e|^2 (per frame lane)
        {
          L yr, yi;
          LN::split(ys[e * TC::YP + q], yr, yi);
          if (ragged) {
            yr = LN::keep(yr, n0, Np);
            yi = LN::keep(yi, n0, Np);
          }
          const L d2 = vfma(yr, yr, yi * yi);
#pragma unroll
          for (int i = 0; i < I; ++i) accd[i] = vfma(wi[i], d2, accd[i]);
        }
#pragma unroll
        for (int k = 0; k < SL; ++k) {
          const VY xu = ys[sr[k] * TC::YP + q];
          const VY yu = ys[sc[k] * TC::YP + q];
#pragma unroll
          for (int fr = 0; fr < FU; ++fr) {
            if (ragged && n0 + fr >= Np) continue;
            const cpx<T> x = yframe(xu, fr), y = yframe(yu, fr);
            const T pr = fma(x.re, y.re, x.im * y.im);   // re(y_r conj(y_c))
            const T pi = fma(x.im, y.re, -(x.re * y.im)); // im(y_r conj(y_c))
#pragma unroll
            for (int i = 0; i < I; ++i) {
              T wf;
              if constexpr (sizeof(T) == 4) wf = fr == 0 ? wi[i].v.x : wi[i].v.y;
              else wf = wi[i].v;
              acco[k][i] = fma2(wf, pr, pi, acco[k][i]);
            }
          }
        }
      }
    }
    seg_new = false;
    consumer_release(pp, t);

    // FP32: the plain sums are flushed into the slot every 2 kFlushUnits
    // units per thread (a flush reduces all I^3 sums of the group: twice the
    // interval of the other passes halves its cost); every lane of the group
    // takes the same tile trips
    const bool flush = sizeof(T) == 4 && !it.seg_end && ++ntile == 2 * flush_tiles(TC::T / IG);
    if (it.seg_end || flush) {
      const int slot = rl.vb - pt.first_block(f);
      double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * (I * I * I);
      T h[BE::NVT], l[BE::NVT];
#pragma unroll
      for (int i = 0; i < I; ++i) {
        if constexpr (sizeof(T) == 4) {
          h[i] = accd[i].v.x + accd[i].v.y;  // the two frame lanes
          l[i] = 0.f;
        } else {
          h[i] = accd[i].v;
          l[i] = 0;
        }
#pragma unroll
        for (int k = 0; k < SL; ++k) {
          h[I + k * 2 * I + 2 * i] = acco[k][i].x;
          h[I + k * 2 * I + 2 * i + 1] = acco[k][i].y;
          l[I + k * 2 * I + 2 * i] = 0;
          l[I + k * 2 * I + 2 * i + 1] = 0;
        }
      }
      // the lanes with the same e (offsets I, 2 I, ... within the warp), in
      // plain arithmetic; the warps' sums then compensated, as GroupReduce
#pragma unroll
      for (int v = 0; v < BE::NVT; ++v) h[v] += l[v];
#pragma unroll
      for (int off = I; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < BE::NVT; ++v) h[v] += __shfl_xor_sync(0xffffffffu, h[v], off);
      if (lane < I) {
        const int nv = lane < I - 1 ? BE::NVT : I;
#pragma unroll
        for (int v = 0; v < BE::NVT; ++v)
          if (v < nv) Red::one(red)[rl.cwarp][BE::red_index(lane, v)] = h[v];
      }
      consumer_sync(rl.group);
      for (int x = tid; x < I * I * I; x += kConsumers) {
        T sh = Red::one(red)[0][x];
        T sl = (T)0;
#pragma unroll
        for (int w2 = 1; w2 < kConsumerWarps; ++w2) {
          if constexpr (sizeof(T) == 4) df_add(sh, sl, Red::one(red)[w2][x], (T)0);
          else sh += Red::one(red)[w2][x];
        }
        const double xv = (double)sh + (double)sl;
        double& o = out[BE::out_index(x)];
        o = flushed ? o + xv : xv;
      }
      consumer_sync(rl.group);
      ntile = 0;
      if (flush) {
#pragma unroll
        for (int i = 0; i < I; ++i) {
          accd[i] = LN::bc(0);
#pragma unroll
          for (int k = 0; k < SL; ++k) acco[k][i] = T2{0, 0};
        }
        flushed = true;
      } else {
        flushed = false;
        seg_new = true;
      }
    }
  }
}

// -------------------------------------------------------------- pass B
// V_i(f) partial sums: sum_n r_i y y^H with r_i = 1/sigma_i from the new v and
// Lambda (Eq. FPI); y y^H packed as the real diagonal, then (re, im) of the
// entries above it in row order.
template <typename T, int I, int J>
__global__ void __maxnreg__((WcovGroups<T, I, J>::value == 2 ? 128 : 255)) k_wcov(FastArgs a) {
  using VY = typename Vec<T>::Y;
  using VV = typename Vec<T>::V;
  using LN = Lane<T>;
  using L = typename LN::L;
  constexpr int G = WcovGroups<T, I, J>::value;
  using TC = Tile<T, I, J, G>;
  constexpr int FU = Vec<T>::FU;
  constexpr int I2 = I * I;
  constexpr int NV = I * I2;
  using Red = GroupReduce<T, NV, (I > 4 ? 1 : 2)>;

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ typename Red::Smem red_all[G];
  __shared__ int aborts[G];
  using PB = ParamsB<T, I, J>;

  const Role rl = role<G>();
  volatile int* abort = &aborts[rl.group];
  typename Red::Smem& red = red_all[rl.group];
  const Partition pt = a.part;
  const long long u0 = pt.block_start(rl.vb);
  const long long u1 = pt.block_start(rl.vb + 1);
  const long long row = a.ld / FU;
  const Pipe<TC::S> pp = setup_pipe<G, TC::S>(smem, TC::STAGE, rl.group, aborts);

  if (!rl.consumer) {  // the whole warp: its lanes finalise pass A's sums in parallel
    produce<T, I, J, true, G>(a, pp, u0, u1, row, rl.vb, abort);
    return;
  }

  if constexpr (I > 4) {
    wcov_consume_big<T, I, J, Red, TC::S, G>(a, pp, u0, u1, rl, abort, red);
  } else {
    const int tid = rl.ctid;
    L lam[J][I];
    // FP32: Kahan-compensated sums (KSum, folded once per tile trip); with
    // I^3 > 32 sums one plain float per value instead (both frames of a unit
    // go into it), which keeps them in registers.  FP64: plain sums.
    constexpr bool kNarrow = sizeof(T) == 4 && NV > 32;
    constexpr bool kComp = sizeof(T) == 4 && !kNarrow;
    using A = std::conditional_t<kNarrow, float, std::conditional_t<kComp, KSum, L>>;
    A acc[NV];

    TileIter it(u0, u1, pt, TC::T, true);
    bool seg_new = true;
    int nseg = 0;          // reductions so far (reduction buffer parity)
    int ntile = 0;         // tile trips since the segment's start or last flush
    int nfold = 0;         // tile trips since the last Kahan step
    bool flushed = false;  // the segment has flushed into its slot
    for (int t = 0; it.next(); ++t) {
      const int f = it.f;
      if (seg_new) {
  #pragma unroll
        for (int q = 0; q < NV; ++q) {
          if constexpr (kNarrow) acc[q] = 0.f;
          else if constexpr (kComp) acc[q].zero();
          else acc[q] = LN::bc(0);
        }
      }
      const int Np = pt.frames(f);
      if (consumer_acquire(a, pp, t, f, abort)) {
        const unsigned char* st = pp.smem + (size_t)(t % TC::S) * TC::STAGE;
        if (seg_new) {  // the new Lambda(f) arrived with the tile
          const PB& sp = *reinterpret_cast<const PB*>(st + TC::ROFF);
  #pragma unroll
          for (int j = 0; j < J; ++j)
  #pragma unroll
            for (int i = 0; i < I; ++i) lam[j][i] = LN::bc(sp.lam[j][i]);
        }
        const VY* ys = reinterpret_cast<const VY*>(st);
        const VV* vs = reinterpret_cast<const VV*>(st + TC::VOFF);
  #pragma unroll 1
        for (int q = tid; q < it.n; q += kConsumers) {
          const int k = it.k + q;
          const int n0 = k * FU;
          if (n0 >= Np) continue;
          L yre[I], yim[I], nyre[I], vv[J];
  #pragma unroll
          for (int m = 0; m < I; ++m) {
            LN::split(ys[m * TC::YP + q], yre[m], yim[m]);
            nyre[m] = yre[m] * LN::bc(-1);
          }
  #pragma unroll
          for (int j = 0; j < J; ++j) vv[j] = LN::real(vs[j * TC::T + q]);
          L w[I];
  #pragma unroll
          for (int i = 0; i < I; ++i) {
            L sg = vv[0] * lam[0][i];
  #pragma unroll
            for (int j = 1; j < J; ++j) sg = vfma(vv[j], lam[j][i], sg);
            w[i] = vrcp(sg);
          }
          if (n0 + FU > Np) {  // the ragged last unit: drop the frames beyond N
  #pragma unroll
            for (int i = 0; i < I; ++i) w[i] = LN::keep(w[i], n0, Np);
  #pragma unroll
            for (int m = 0; m < I; ++m) {
              yre[m] = LN::keep(yre[m], n0, Np);
              yim[m] = LN::keep(yim[m], n0, Np);
              nyre[m] = LN::keep(nyre[m], n0, Np);
            }
          }
          // each packed entry of y y^H, then at once its I weighted sums (the
          // entry is live for one step only)
          auto add = [&](int mm, L x) {
  #pragma unroll
            for (int i = 0; i < I; ++i) {
              if constexpr (kNarrow)
                acc[i * I2 + mm] = fmaf(w[i].v.y, x.v.y, fmaf(w[i].v.x, x.v.x, acc[i * I2 + mm]));
              else if constexpr (kComp)
                acc[i * I2 + mm].p = fmaf(w[i].v.y, x.v.y, fmaf(w[i].v.x, x.v.x, acc[i * I2 + mm].p));
              else
                acc[i * I2 + mm] = vfma(w[i], x, acc[i * I2 + mm]);
            }
          };
          int m = I;
  #pragma unroll
          for (int rr = 0; rr < I; ++rr) {
            add(rr, vfma(yre[rr], yre[rr], yim[rr] * yim[rr]));
  #pragma unroll
            for (int c = rr + 1; c < I; ++c) {
              add(m, vfma(yre[rr], yre[c], yim[rr] * yim[c]));           // re(y_r conj(y_c))
              add(m + 1, vfma(nyre[rr], yim[c], yim[rr] * yre[c]));      // im(y_r conj(y_c))
              m += 2;
            }
          }
        }
        if constexpr (kComp) {  // one Kahan step every kFoldTiles tile trips
          if (++nfold == kFoldTiles) {
            nfold = 0;
  #pragma unroll
            for (int q = 0; q < NV; ++q) acc[q].fold();
          }
        }
      }

      seg_new = false;
      consumer_release(pp, t);

      // plain FP32 sums (kNarrow) are flushed into the slot every
      // kFlushUnits units per thread (as in pass A)
      const bool flush = kNarrow && !it.seg_end && ++ntile == flush_tiles(TC::T / kConsumers);
      if (it.seg_end || flush) {
        const int slot = rl.vb - pt.first_block(f);
        double* out = a.part_buf + ((size_t)f * pt.max_slots + slot) * NV;
        if constexpr (kNarrow) {
          Red::run(acc, red, out, rl, nseg, flushed);
        } else if constexpr (kComp) {
          float hi[NV];
  #pragma unroll
          for (int q = 0; q < NV; ++q) hi[q] = acc[q].value();
          Red::run(hi, red, out, rl, nseg);
        } else {
          double hi[NV];
  #pragma unroll
          for (int q = 0; q < NV; ++q) hi[q] = acc[q].v;
          Red::run(hi, red, out, rl, nseg);
        }
        ++nseg;  // the next reduction goes through the other buffer
        ntile = 0;
        if (flush) {
          if constexpr (kNarrow) {
  #pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = 0.f;
          }
          flushed = true;
        } else {
          flushed = false;
          seg_new = true;
        }
      }
    }
  }
}

}  // namespace ffca
