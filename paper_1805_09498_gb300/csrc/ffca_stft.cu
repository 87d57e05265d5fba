// STFT front end and inverse (overlap-add) back end with the parameters of
// the paper's experiments (Table 1: frame length L = 1024, shift H = 512,
// square root of the Hann window; bins up to the Nyquist frequency, F = 513,
// Sec. 2).  The frame's 1024 real samples are transformed as one 512-point
// complex FFT of z(t) = x(2t) + i x(2t+1), then split into the spectrum of
// the real frame:
//     X[k] = E[k] + e^{-2 pi i k/1024} O[k],  E[k] = (Z[k] + conj Z[512-k]) / 2,
//     O[k] = (Z[k] - conj Z[512-k]) / (2i),   k = 0 .. 512 (Z[512] = Z[0]).
// The inverse runs the same steps backwards.  FP32 data, twiddles and window
// rounded from FP64 values computed on the host.
//
// One warp transforms one frame (fft512_warp: 512 = 16 x 32, a 16-point DFT
// per lane, one transpose through the warp's shared-memory buffer, then a
// radix-2 step and a second 16-point DFT per lane), so no barrier separates
// the stages and no value crosses lanes by shuffles.  The real split pairs
// bins k and 512 - k (one pair of reads makes both).  Both directions run
// persistent CTAs of kFrames warps over groups of kFrames frames: the next
// group's input is copied into a second shared-memory stage (cp.async)
// while the current group is transformed.  The spectra move through shared
// memory with swizzled bin rows (conflict-free per-bin stores, 16-byte
// loads) as runs of kFrames frames per bin: the frame-contiguous mic-planar
// layout, 64 bytes per bin row, two frames per 16-byte store.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "ffca.h"

namespace {

constexpr int kL = 1024;        // frame length
constexpr int kH = 512;         // frame shift
constexpr int kM = 512;         // complex FFT size (two real samples per point)
constexpr int kF = kL / 2 + 1;  // bins up to Nyquist
constexpr int kFrames = 8;      // frames per group: one per warp of a CTA (about 100 KB of shared memory: two CTAs per SM)
constexpr int kThreads = 32 * kFrames;
constexpr int kMaxDev = 64;

__device__ float2 g_tw512[kM];   // e^{-2 pi i m / 512}
__device__ float2 g_tw1024[kF];  // e^{-2 pi i k / 1024}, k = 0 .. 512
__constant__ float2 c_w32[32];   // e^{-2 pi i m / 32}: indexed by compile-time constants only (operands of the
                                 // arithmetic, no loads); W16^m = W32^(2m)
__device__ __align__(16) float g_win[kL];  // sin(pi t / 1024): the square root of the periodic Hann window

std::mutex g_tab_mutex;
bool g_tab_ready[kMaxDev];

// Fill the tables of the current device once (FP64 values rounded to FP32).
ffca_status ensure_tables() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return FFCA_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_tab_mutex);
  if (g_tab_ready[dev]) return FFCA_OK;
  static float2 tw512[kM], tw1024[kF], w32[32];
  static float win[kL];
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < kM; ++m)
    tw512[m] = make_float2((float)std::cos(2.0 * pi * m / kM), (float)-std::sin(2.0 * pi * m / kM));
  for (int k = 0; k < kF; ++k)
    tw1024[k] = make_float2((float)std::cos(2.0 * pi * k / kL), (float)-std::sin(2.0 * pi * k / kL));
  for (int t = 0; t < kL; ++t) win[t] = (float)std::sin(pi * t / kL);
  for (int m = 0; m < 32; ++m) w32[m] = make_float2((float)std::cos(2.0 * pi * m / 32), (float)-std::sin(2.0 * pi * m / 32));
  if (cudaMemcpyToSymbol(g_tw512, tw512, sizeof(tw512)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_tw1024, tw1024, sizeof(tw1024)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_win, win, sizeof(win)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_w32, w32, sizeof(w32)) != cudaSuccess)
    return FFCA_ERR_CUDA;
  g_tab_ready[dev] = true;
  return FFCA_OK;
}

__device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ inline float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

// 4-point DFT (forward: e^{-2 pi i q r / 4}).
// The sums and differences of whole complex values as paired FP32
// operations (one f32x2 instruction each); the -i rotation of the odd
// outputs in plain FP32.
__device__ inline float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ inline float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ inline void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  a1 = make_float2(t1.x + d.y, t1.y - d.x);  // t1 + (-i) d
  a3 = make_float2(t1.x - d.y, t1.y + d.x);  // t1 - (-i) d
}

// 16-point DFT of u[0..15] in registers (forward): with n = 4 n1 + n2 and
// k = k1 + 4 k2, X[k] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) u[4 n1 + n2]:
// four 4-point DFTs over n1, the twiddles W16^(n2 k1) (constant operands:
// W16^m = W32^(2m)), four 4-point DFTs over n2.  Output in natural order.
__device__ inline void dft16(float2 (&u)[16]) {
  float2 y[4][4];  // [n2][k1]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a0 = u[n2], a1 = u[4 + n2], a2 = u[8 + n2], a3 = u[12 + n2];
    dft4(a0, a1, a2, a3);
    y[n2][0] = a0;
    y[n2][1] = a1;
    y[n2][2] = a2;
    y[n2][3] = a3;
  }
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = cmul(y[n2][k1], c_w32[2 * n2 * k1]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4(a0, a1, a2, a3);
    u[k1] = a0;
    u[k1 + 4] = a1;
    u[k1 + 8] = a2;
    u[k1 + 12] = a3;
  }
}

// Per-warp work buffer: the transpose of fft512_warp (32 rows of 16 values,
// pitch 17, so that the lanes' row writes fall in distinct banks), then the
// 512 values of Z (forward) or the frame's two windowed halves (inverse).
constexpr int kBufPitch = 17;
constexpr int kBuf = 32 * kBufPitch;

// 512-point forward DFT by one warp.  Lane l enters with u[q] = z[l + 32 q]
// (q = 0..15).  With k = r + 16 k2 (r = 0..15, k2 = 0..31):
//   Z[r + 16 k2] = sum_l W32^(l k2) a_l[r],  a_l[r] = W512^(l r) sum_q W16^(q r) z[l + 32 q].
// Every lane forms its a_l (dft16 and its twiddles tw1[r - 1] = W512^(l r),
// held in registers by the caller) and writes it to row l of the buffer.
// Lane L then takes r = L mod 16 and g = L / 16 and splits the 32-point DFT
// over l by the parity of k2 = 2 j + g (decimation in frequency):
// Z[r + 16 (2 j + g)] = sum_{m<16} W16^(m j) W32^(m g) (a_m[r] + (-1)^g a_{m+16}[r]),
// a 16-point DFT of sixteen values it reads from the buffer.  On return lane
// L holds u[j] = Z[r + 16 (2 j + g)] = Z[L + 32 j], and the buffer is free.
__device__ inline void fft512_warp(float2 (&u)[16], int lane, float2* __restrict__ buf, const float2 (&tw1)[15]) {
  dft16(u);
#pragma unroll
  for (int r = 1; r < 16; ++r) u[r] = cmul(u[r], tw1[r - 1]);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[lane * kBufPitch + r] = u[r];
  __syncwarp();
  const int r = lane & 15;
  const bool odd = lane >= 16;  // g = 1
  const float sgn = odd ? -1.f : 1.f;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const float2 p = buf[m * kBufPitch + r], q = buf[(m + 16) * kBufPitch + r];
    u[m] = __ffma2_rn(make_float2(sgn, sgn), q, p);
  }
#pragma unroll
  for (int m = 1; m < 16; ++m) {  // W32^(m g)
    const float2 t = cmul(u[m], c_w32[m]);
    u[m] = odd ? t : u[m];
  }
  __syncwarp();
  dft16(u);
}

// The first-stage twiddles of lane l, W512^(l r) for r = 1..15.
__device__ inline void lane_twiddles(int lane, float2 (&tw1)[15]) {
#pragma unroll
  for (int r = 1; r < 16; ++r) tw1[r - 1] = __ldg(g_tw512 + ((lane * r) & (kM - 1)));
}

// The spectra of a CTA's frames, bin-major: row k holds the kFrames frames
// of bin k, frame w at position w ^ swz(k).  The swizzle spreads a warp's
// stores of one frame's 32 consecutive bins over all banks (two wavefronts
// for 64-bit stores) and keeps every pair of frames (2p, 2p + 1) in one
// aligned 16-byte slot (in swapped order when swz(k) is odd), so that the
// rows leave in 16-byte loads and stores.
__device__ inline int swz(int k) { return (k >> 1) & (kFrames - 1); }

// Samples of a CTA's group of kFrames frames: frames n0 .. n0 + 7 span
// (kFrames + 1) H consecutive samples.
constexpr int kGroupSamples = (kFrames + 1) * kH;

// Shared memory of one CTA.
struct StftSmem {
  float2 buf[kFrames][kBuf];  // each warp's work buffer
  float2 spec[kF][kFrames];   // the CTA's spectra (swizzled rows)
};
// Forward: two stages of input samples besides.
struct StftFwdSmem {
  StftSmem s;
  float x[2][kGroupSamples];
};
// The inverse keeps its frame's two windowed halves in the warp's buffer.
static_assert(kBuf * sizeof(float2) >= 2 * kH * sizeof(float), "halves fit in the buffer");
static_assert((kBuf * sizeof(float2)) % 16 == 0 && sizeof(StftSmem) % 16 == 0, "16-byte alignment");

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ inline void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
// 8 bytes from src, or zeros (nothing read) when !valid
__device__ inline void cp_async8z(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// x [C][S] float -> out [C][F][ld] complex64 (frames 0 .. N-1, then zero to
// ld).  Persistent: a CTA takes the groups of kFrames frames it = blockIdx.x,
// blockIdx.x + gridDim.x, ... of the C x ceil(N / kFrames) groups (channel
// it / G, frames kFrames (it mod G) ..), and copies the next group's samples
// into the other input stage (cp.async) while it transforms this one; warp
// w transforms frame w of the group.  VEC: x and S allow 16-byte copies.
template <bool VEC>
__global__ void __launch_bounds__(kThreads, 2) k_stft(const float* __restrict__ x, int C, long long S, int N,
                                                      float2* __restrict__ out, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftFwdSmem& sm = *reinterpret_cast<StftFwdSmem*>(smem_raw);
  const int G = (N + kFrames - 1) / kFrames, items = C * G;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // copy the samples of group `item` into stage st
  auto fetch = [&](int item, int st) {
    const int c = item / G, n0 = (item % G) * kFrames, nf = min(kFrames, N - n0);
    const float* src = x + (size_t)c * S + (size_t)n0 * kH;
    const int len = (nf + 1) * kH;  // samples, a multiple of 512
    if (VEC) {
      for (int t = threadIdx.x; t < len / 4; t += kThreads) cp_async16(sm.x[st] + 4 * t, src + 4 * t);
    } else {
      for (int t = threadIdx.x; t < len; t += kThreads) cp_async4(sm.x[st] + t, src + t);
    }
  };
  int it = blockIdx.x;
  if (it >= items) return;
  float2 tw1[15];
  lane_twiddles(lane, tw1);
  const float2 wl = __ldg(g_tw1024 + lane);  // W1024^l
  fetch(it, 0);
  cp_async_commit();
  for (int st = 0; it < items; it += gridDim.x, st ^= 1) {
    if (it + (int)gridDim.x < items) fetch(it + gridDim.x, st ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this group's copies (all but the newest group) have landed
    __syncthreads();
    const int c = it / G, n0 = (it % G) * kFrames, nf = min(kFrames, N - n0);
    if (w < nf) {
      const float2* xf = reinterpret_cast<const float2*>(sm.x[st] + w * kH);  // frame n0 + w
      const float2* win = reinterpret_cast<const float2*>(g_win);
      float2 u[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {  // z(t) = w(2t) x(2t) + i w(2t+1) x(2t+1), t = l + 32 q
        const int t = lane + 32 * q;
        const float2 xv = xf[t], wv = __ldg(win + t);
        u[q] = make_float2(wv.x * xv.x, wv.y * xv.y);
      }
      float2* zb = sm.s.buf[w];
      fft512_warp(u, lane, zb, tw1);
#pragma unroll
      for (int j = 0; j < 16; ++j) zb[lane + 32 * j] = u[j];  // Z[k] at k
      __syncwarp();
      // X[k] = E + W1024^k O and X[512 - k] = conj(E - W1024^k O), with
      // E = (Z[k] + conj Z[512-k]) / 2, O = (Z[k] - conj Z[512-k]) / (2i), k = 0 .. 256
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int k = lane + 32 * i;
        if (i < 8 || k == kM / 2) {
          const float2 zk = zb[k];
          const float2 zm = cconj(zb[(kM - k) & (kM - 1)]);
          const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
          const float2 o = mul_mi(make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y - zm.y)));
          const float2 t = cmul(cmul(wl, c_w32[i]), o);  // W1024^k = W1024^l W32^i
          sm.s.spec[k][w ^ swz(k)] = cadd(e, t);
          if (k < kM / 2) sm.s.spec[kL / 2 - k][w ^ swz(kL / 2 - k)] = cconj(csub(e, t));
        }
      }
    }
    __syncthreads();
    // runs of consecutive frames per bin, two frames per 16-byte store
    float2* oc = out + (size_t)c * kF * ld;
    {
      // thread t stores frames n, n + 1 (n = 2 (t mod 4)) of the bins f0 + 64 i (f0 = t / 4); swz(f0 + 64 i) = swz(f0)
      constexpr int kPairs = kFrames / 2, kRows = kThreads / kPairs;
      const int n = 2 * (threadIdx.x % kPairs), f0 = threadIdx.x / kPairs, sw = swz(f0);
      const float4* srow = reinterpret_cast<const float4*>(&sm.s.spec[f0][(n ^ sw) & ~1]);
      float2* dst = oc + (size_t)f0 * ld + n0 + n;
      if (n < nf) {
#pragma unroll
        for (int i = 0; i < (kF + kRows - 1) / kRows; ++i) {
          if (f0 + i * kRows < kF) {
            const float4 v = srow[i * kRows * kFrames / 2];
            const float2 a = (sw & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);   // frame n
            const float2 b2 = (sw & 1) ? make_float2(v.x, v.y) : make_float2(v.z, v.w);  // frame n + 1
            if (n + 1 < nf) *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b2.x, b2.y);
            else *dst = a;
          }
          dst += (size_t)kRows * ld;
        }
      }
    }
    // padding frames N .. ld - 1 of each row: written with the channel's last group
    if (n0 + kFrames >= N) {
      const int pad = ld - N;
      for (int t = threadIdx.x; t < kF * pad; t += kThreads) {
        const int f = t / pad, n = N + t % pad;
        oc[(size_t)f * ld + n] = make_float2(0.f, 0.f);
      }
    }
  }
  cp_async_wait<0>();
}

// One frame's inverse by a warp: the spectrum X[k] = x_of(k), k = 0 .. 512,
// to the frame's 1024 windowed samples, left in the warp's buffer as pairs
// (zeros where !on).  Z[k] = E[k] + i O[k] from X[k] and X[512 - k] (bins 0
// and L/2 of a real signal's spectrum are real: their imaginary parts are
// ignored), conjugated for the forward transform:
// IDFT(Z) = conj(DFT(conj Z)) / 512.
template <typename X>
__device__ inline void inverse_frame(X x_of, bool on, int lane, float2* __restrict__ buf, const float2 (&tw1)[15],
                                     float2 wl) {
  float2 u[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int k = lane + 32 * q;
    float2 xk = x_of(k);
    float2 xm = cconj(x_of(kM - k));
    if (k == 0) {
      xk.y = 0.f;
      xm.y = 0.f;
    }
    const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y + xm.y));
    const float2 o = cmul(make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y - xm.y)), cconj(cmul(wl, c_w32[q])));
    u[q] = cconj(make_float2(e.x - o.y, e.y + o.x));
  }
  fft512_warp(u, lane, buf, tw1);  // lane l: DFT(conj Z) at t = l + 32 j in u[j]
  const float2* win = reinterpret_cast<const float2*>(g_win);
  const float sc = 1.0f / kM;
#pragma unroll
  for (int j = 0; j < 16; ++j) {  // x(2t) = Re / 512, x(2t+1) = -Im / 512, windowed
    const int t = lane + 32 * j;
    const float2 wv = __ldg(win + t);
    buf[t] = on ? make_float2(wv.x * u[j].x * sc, -wv.y * u[j].y * sc) : make_float2(0.f, 0.f);
  }
}

// in [C][F][ld] complex64 (frames 0 .. N-1) -> out [C][(N + 1) H] float.
// Output block k (samples k H .. k H + H - 1, k = 0 .. N) is the second half
// of frame k - 1 plus the first half of frame k.  Group b of a channel holds
// the blocks and the frames 8 b .. 8 b + 7: warp w inverts frame 8 b + w
// (a missing frame adds nothing), and block 8 b + w adds its first half to
// the second half of frame 8 b + w - 1, which for w = 0 is the last frame of
// group b - 1.  Persistent CTAs take contiguous ranges of the
// C x ceil((N + 1) / 8) groups and carry that half from one group to the
// next (two alternating buffers; zeros at a channel's first group); at the
// start of a range with b > 0, warp 0 first inverts frame 8 b - 1 for it.
// The next group's spectra (runs of 8 frames per bin, zeros beyond N) are
// copied into the other input stage (cp.async) while this group is
// transformed.  VEC: out allows 16-byte stores.
struct StftInvSmem {
  float2 buf[kFrames][kBuf];
  float2 in[2][kF][kFrames];  // swizzled rows, as the forward's spectra
  float carry[2][kH];         // second half of the frame before the group
  float2 pro[kF];             // the spectrum of the frame before a range's first group
};

template <bool VEC>
__global__ void __launch_bounds__(kThreads, 2) k_istft(const float2* __restrict__ in, int C, int N, int ld,
                                                       float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftInvSmem& sm = *reinterpret_cast<StftInvSmem*>(smem_raw);
  const int B = (N + kFrames) / kFrames, items = C * B;
  const int per = (items + (int)gridDim.x - 1) / (int)gridDim.x;
  const int it0 = blockIdx.x * per, it1 = min(items, it0 + per);
  if (it0 >= it1) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto fetch = [&](int item, int st) {
    const int c = item / B, m0 = (item % B) * kFrames;
    const float2* ic = in + (size_t)c * kF * ld;
    // thread t copies frame fr = t mod 8 of the bins f0 + 32 i (f0 = t / 8); swz(f0 + 32 i) = swz(f0)
    const int fr = threadIdx.x % kFrames, f0 = threadIdx.x / kFrames, m = m0 + fr;
    const bool ok = m < N;
    const float2* src = ok ? ic + (size_t)f0 * ld + m : ic;
    const size_t step = ok ? (size_t)(kThreads / kFrames) * ld : 0;
    float2* dst = &sm.in[st][f0][fr ^ swz(f0)];
#pragma unroll
    for (int i = 0; i < (kF + kThreads / kFrames - 1) / (kThreads / kFrames); ++i) {
      if (f0 + i * (kThreads / kFrames) < kF) cp_async8z(dst, src, ok);
      src += step;
      dst += (kThreads / kFrames) * kFrames;
    }
  };
  float2 tw1[15];
  lane_twiddles(lane, tw1);
  const float2 wl = __ldg(g_tw1024 + lane);  // W1024^l
  fetch(it0, 0);
  cp_async_commit();
  {  // the carried half before the range's first group
    const int c0 = it0 / B, b0 = it0 % B;
    if (b0 > 0) {
      const float2* col = in + (size_t)c0 * kF * ld + (kFrames * b0 - 1);  // frame 8 b0 - 1 < N
      for (int t = threadIdx.x; t < kF; t += kThreads) sm.pro[t] = __ldg(col + (size_t)t * ld);
      __syncthreads();
      if (w == 0) {
        inverse_frame([&](int k) { return sm.pro[k]; }, true, lane, sm.buf[0], tw1, wl);
        __syncwarp();
        const float* h = reinterpret_cast<const float*>(sm.buf[0]);
        for (int t = lane; t < kH; t += 32) sm.carry[0][t] = h[kH + t];
      }
    }
  }
  int par = 0;  // the carry buffer of the current group
  for (int it = it0, st = 0; it < it1; ++it, st ^= 1) {
    if (it + 1 < it1) fetch(it + 1, st ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int c = it / B, b = it % B, m = kFrames * b + w;
    inverse_frame([&](int k) { return sm.in[st][k][w ^ swz(k)]; }, m < N, lane, sm.buf[w], tw1, wl);
    __syncthreads();
    // blocks 8 b + kk: second half of frame 8 b + kk - 1 (the carry for kk = 0, none at b = 0)
    // plus the first half of frame 8 b + kk
    float* oc = out + (size_t)c * ((size_t)N + 1) * kH + (size_t)kFrames * b * kH;
    const int nk = min(kFrames, N + 1 - kFrames * b);
    const bool first = b == 0;
    if (VEC) {
      for (int t = threadIdx.x; t < nk * (kH / 4); t += kThreads) {
        const int kk = t / (kH / 4), s4 = t % (kH / 4);
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kk > 0) a = reinterpret_cast<const float4*>(sm.buf[kk - 1])[kH / 4 + s4];
        else if (!first) a = reinterpret_cast<const float4*>(sm.carry[par])[s4];
        const float4 b2 = reinterpret_cast<const float4*>(sm.buf[kk])[s4];
        reinterpret_cast<float4*>(oc + (size_t)kk * kH)[s4] = make_float4(a.x + b2.x, a.y + b2.y, a.z + b2.z, a.w + b2.w);
      }
    } else {
      for (int t = threadIdx.x; t < nk * kH; t += kThreads) {
        const int kk = t / kH, s1 = t % kH;
        float a = 0.f;
        if (kk > 0) a = reinterpret_cast<const float*>(sm.buf[kk - 1])[kH + s1];
        else if (!first) a = sm.carry[par][s1];
        oc[(size_t)kk * kH + s1] = a + reinterpret_cast<const float*>(sm.buf[kk])[s1];
      }
    }
    // the next group's carry: the second half of frame 8 b + 7
    {
      const float* h = reinterpret_cast<const float*>(sm.buf[kFrames - 1]);
      for (int t = threadIdx.x; t < kH; t += kThreads) sm.carry[par ^ 1][t] = h[kH + t];
    }
    par ^= 1;
  }
  cp_async_wait<0>();
}

// Persistent grid: as many CTAs as are resident at once, at most one per work item.
template <typename K>
int resident_grid(K kernel, size_t smem, long long items) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, smem) != cudaSuccess || per < 1)
    return 0;
  return (int)std::min<long long>(items, (long long)sms * per);
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

ffca_status ffca_stft(const float* x, int C, long long S, void* out, int ld, void* stream) {
  if (C < 0 || S < 0 || ld < 0) return FFCA_ERR_ARG;
  const long long Nl = S >= kL ? 1 + (S - kL) / kH : 0;
  if (Nl > (1 << 30)) return FFCA_ERR_ARG;
  const int N = (int)Nl;
  if (C == 0 || N == 0) return FFCA_OK;
  const long long items = (long long)C * ((N + kFrames - 1) / kFrames);
  if (ld < N || (ld % 4) != 0 || !x || !out || (reinterpret_cast<uintptr_t>(out) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(x) % 4) != 0 || C > 65535 || items > INT32_MAX / 2)
    return FFCA_ERR_ARG;
  ffca_status st = ensure_tables();
  if (st != FFCA_OK) return st;
  const size_t smem = sizeof(StftFwdSmem);
  const bool vec = (reinterpret_cast<uintptr_t>(x) % 16) == 0 && (S % 4) == 0;
  auto kern = vec ? k_stft<true> : k_stft<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FFCA_ERR_CUDA;
  const int grid = resident_grid(kern, smem, items);
  if (grid < 1) return FFCA_ERR_CUDA;
  kern<<<grid, kThreads, smem, as_stream(stream)>>>(x, C, S, N, static_cast<float2*>(out), ld);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

ffca_status ffca_istft(const void* in, int C, int N, int ld, float* out, void* stream) {
  if (C < 0 || N < 0 || ld < 0) return FFCA_ERR_ARG;
  if (C == 0 || N == 0) return FFCA_OK;
  const long long items = (long long)C * ((N + kFrames) / kFrames);
  if (ld < N || !in || !out || (reinterpret_cast<uintptr_t>(in) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(out) % 4) != 0 || C > 65535 || N > (1 << 30) - 2 || items > INT32_MAX / 2)
    return FFCA_ERR_ARG;
  ffca_status st = ensure_tables();
  if (st != FFCA_OK) return st;
  const size_t smem = sizeof(StftInvSmem);
  auto kern = (reinterpret_cast<uintptr_t>(out) % 16) == 0 ? k_istft<true> : k_istft<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FFCA_ERR_CUDA;
  const int grid = resident_grid(kern, smem, items);
  if (grid < 1) return FFCA_ERR_CUDA;
  kern<<<grid, kThreads, smem, as_stream(stream)>>>(static_cast<const float2*>(in), C, N, ld, out);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

}  // extern "C"
