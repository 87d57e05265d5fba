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
// One warp transforms one frame, in registers and across its lanes by
// shuffles (fft512_warp: 512 = 16 x 32, a 16-point DFT per lane and a
// 32-point DFT over the lanes), so no barrier separates the stages; a CTA
// takes kFrames consecutive frames of one channel and moves the spectra
// through shared memory as runs of kFrames frames per bin (the
// frame-contiguous mic-planar layout), 64 bytes per bin row.  Sixteen frames
// per CTA (128-byte runs) measured no faster forward and slower inverse
// (2.45 against 1.71 ms): their 135 KB of shared memory leave one CTA per SM,
// whose load, transform and store phases then do not overlap another's.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "ffca.h"

namespace {

constexpr int kL = 1024;        // frame length
constexpr int kH = 512;         // frame shift
constexpr int kM = 512;         // complex FFT size (two real samples per point)
constexpr int kF = kL / 2 + 1;  // bins up to Nyquist
constexpr int kFrames = 8;      // frames per CTA: one per warp (68 KB of shared memory: three CTAs per SM)
constexpr int kThreads = 32 * kFrames;
constexpr int kMaxDev = 64;

__device__ float2 g_tw512[kM];   // e^{-2 pi i m / 512}
__device__ float2 g_tw1024[kF];  // e^{-2 pi i k / 1024}, k = 0 .. 512
__device__ float g_win[kL];      // sin(pi t / 1024): the square root of the periodic Hann window

std::mutex g_tab_mutex;
bool g_tab_ready[kMaxDev];

// Fill the tables of the current device once (FP64 values rounded to FP32).
ffca_status ensure_tables() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return FFCA_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_tab_mutex);
  if (g_tab_ready[dev]) return FFCA_OK;
  static float2 tw512[kM], tw1024[kF];
  static float win[kL];
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < kM; ++m)
    tw512[m] = make_float2((float)std::cos(2.0 * pi * m / kM), (float)-std::sin(2.0 * pi * m / kM));
  for (int k = 0; k < kF; ++k)
    tw1024[k] = make_float2((float)std::cos(2.0 * pi * k / kL), (float)-std::sin(2.0 * pi * k / kL));
  for (int t = 0; t < kL; ++t) win[t] = (float)std::sin(pi * t / kL);
  if (cudaMemcpyToSymbol(g_tw512, tw512, sizeof(tw512)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_tw1024, tw1024, sizeof(tw1024)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_win, win, sizeof(win)) != cudaSuccess)
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
__device__ inline void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// 16-point DFT of u[0..15] in registers (forward): with n = 4 n1 + n2 and
// k = k1 + 4 k2, X[k] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) u[4 n1 + n2]:
// four 4-point DFTs over n1, the twiddles W16^(n2 k1) (from the 512-point
// table: W16^m = W512^(32 m)), four 4-point DFTs over n2.  Output in
// natural order.
__device__ inline void dft16(float2 (&u)[16], const float2* __restrict__ tw) {
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
    for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = cmul(y[n2][k1], __ldg(tw + 32 * n2 * k1));
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

// 512-point forward DFT by one warp.  Lane l enters with u[q] = z[l + 32 q]
// (q = 0..15).  Writing k = r + 16 k2 (r = 0..15, k2 = 0..31):
//   Z[r + 16 k2] = sum_l W32^(l k2) W512^(l r) sum_q W16^(q r) z[l + 32 q],
// so every lane transforms its sixteen values (dft16), multiplies entry r by
// W512^(l r), and the warp runs the 32-point DFT over l for every r as five
// radix-2 decimation-in-frequency stages across the lanes (partner lane
// l ^ h; the upper lane takes (partner - own) W_2h^(l mod h)).  On return
// lane l holds u[r] = Z[r + 16 rev5(l)], rev5 the 5-bit reversal.
__device__ inline void fft512_warp(float2 (&u)[16], int lane, const float2* __restrict__ tw) {
  dft16(u, tw);
#pragma unroll
  for (int r = 1; r < 16; ++r) u[r] = cmul(u[r], __ldg(tw + ((lane * r) & (kM - 1))));
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const float2 w = __ldg(tw + (lane & (h - 1)) * (256 / h));  // W_2h^(l mod h) = W512^((l mod h) 256 / h)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, u[r].x, h), __shfl_xor_sync(0xffffffffu, u[r].y, h));
      u[r] = upper ? cmul(csub(o, u[r]), w) : cadd(u[r], o);
    }
  }
}

__device__ inline int rev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

// Padded index of Z[k] in a warp's buffer: k mod 16 + 17 (k / 16), so that
// the lanes' writes of u[r] and their reads of consecutive k hit distinct
// banks (up to two-way).
__device__ inline int zpad(int k) { return (k & 15) + 17 * (k >> 4); }
constexpr int kZPad = 17 * (kM / 16);

// Padded index of sample s of a half frame (one float of padding per 32), so
// that the lanes' scalar stores of samples 2t, 2t+1 at t = r + 16 rev5(l)
// fall in distinct banks.
__device__ inline int spad(int s) { return s + (s >> 5); }
constexpr int kHalfPad = kH + kH / 32;

// Shared memory of one CTA.
struct StftSmem {
  float2 z[kFrames][kZPad];        // each warp's Z (forward: the real split reads Z[k], Z[512 - k])
  float2 spec[kF][kFrames];        // the CTA's spectra, bin-major (forward: out; inverse: in)
};
// The inverse keeps the windowed halves of its frames where the forward
// transform keeps Z.
static_assert(sizeof(StftSmem::z) >= 2 * kFrames * kHalfPad * sizeof(float), "halves fit in z");

// x [C][S] float -> out [C][F][ld] complex64 (frames 0 .. N-1, then zero to
// ld).  Warp w of the CTA transforms frame n0 + w of channel blockIdx.y.
__global__ void __launch_bounds__(kThreads) k_stft(const float* __restrict__ x, long long S, int N,
                                                   float2* __restrict__ out, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftSmem& sm = *reinterpret_cast<StftSmem*>(smem_raw);
  const int c = blockIdx.y;
  const int n0 = blockIdx.x * kFrames;
  const int nf = min(kFrames, N - n0);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < nf) {
    const float* xf = x + (size_t)c * S + (size_t)(n0 + w) * kH;  // samples n H .. n H + L - 1 (inside the signal)
    float2 u[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // z(t) = w(2t) x(2t) + i w(2t+1) x(2t+1), t = l + 32 q
      const int t = lane + 32 * q;
      u[q] = make_float2(__ldg(g_win + 2 * t) * __ldg(xf + 2 * t), __ldg(g_win + 2 * t + 1) * __ldg(xf + 2 * t + 1));
    }
    fft512_warp(u, lane, g_tw512);
    float2* zb = sm.z[w];
    const int base = 16 * rev5(lane);
#pragma unroll
    for (int r = 0; r < 16; ++r) zb[zpad(base + r)] = u[r];
    __syncwarp();
    // X[k] = E[k] + W1024^k O[k], E = (Z[k] + conj Z[512-k]) / 2, O = (Z[k] - conj Z[512-k]) / (2i)
    for (int k = lane; k < kF; k += 32) {
      const float2 zk = zb[zpad(k & (kM - 1))];
      const float2 zm = cconj(zb[zpad((kM - k) & (kM - 1))]);
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      const float2 o = mul_mi(make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y - zm.y)));
      sm.spec[k][w] = cadd(e, cmul(__ldg(g_tw1024 + k), o));
    }
  }
  __syncthreads();
  // runs of consecutive frames per bin
  float2* oc = out + (size_t)c * kF * ld;
  for (int t = threadIdx.x; t < kF * kFrames; t += kThreads) {
    const int f = t / kFrames, n = t % kFrames;
    if (n < nf) oc[(size_t)f * ld + n0 + n] = sm.spec[f][n];
  }
  // padding frames N .. ld - 1 of each row: written by the last CTA
  if (n0 + kFrames >= N) {
    const int pad = ld - N;
    for (int t = threadIdx.x; t < kF * pad; t += kThreads) {
      const int f = t / pad, n = N + t % pad;
      oc[(size_t)f * ld + n] = make_float2(0.f, 0.f);
    }
  }
}

// in [C][F][ld] complex64 (frames 0 .. N-1) -> out [C][(N + 1) H] float.  A
// CTA writes the kFrames - 1 output blocks k = k0 .. k0 + kFrames - 2 of H
// samples (k <= N), block k being the second half of frame k - 1 plus the
// first half of frame k: warp w inverts frame m0 + w (m0 = k0 - 1; a missing
// frame adds nothing).  The spectra arrive as runs of kFrames consecutive
// frames per bin (coalesced), staged in spec; the windowed halves go to z.
__global__ void __launch_bounds__(kThreads) k_istft(const float2* __restrict__ in, int N, int ld,
                                                    float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftSmem& sm = *reinterpret_cast<StftSmem*>(smem_raw);
  const int c = blockIdx.y;
  const int k0 = blockIdx.x * (kFrames - 1);
  const int m0 = k0 - 1;  // frames m0 .. m0 + kFrames - 1
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float2* ic = in + (size_t)c * kF * ld;
  for (int t = threadIdx.x; t < kF * kFrames; t += kThreads) {
    const int f = t / kFrames, fr = t % kFrames, m = m0 + fr;
    sm.spec[f][fr] = (m >= 0 && m < N) ? __ldg(ic + (size_t)f * ld + m) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int m = m0 + w;
  const bool on = m >= 0 && m < N;
  float2 u[16];
  // Z[k] = E[k] + i O[k] from X[k] and X[512 - k] (bins 0 and L/2 of a real
  // signal's spectrum are real: their imaginary parts are ignored), conjugated
  // for the forward transform: IDFT(Z) = conj(DFT(conj Z)) / 512
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int k = lane + 32 * q;
    float2 xk = sm.spec[k][w];
    float2 xm = cconj(sm.spec[kM - k][w]);
    if (k == 0) {
      xk.y = 0.f;
      xm.y = 0.f;
    }
    const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y + xm.y));
    const float2 o = cmul(make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y - xm.y)), cconj(__ldg(g_tw1024 + k)));
    u[q] = cconj(make_float2(e.x - o.y, e.y + o.x));
  }
  fft512_warp(u, lane, g_tw512);  // lane l: DFT(conj Z) at t = r + 16 rev5(l)
  float* first = reinterpret_cast<float*>(sm.z);  // [kFrames][kHalfPad]
  float* second = first + kFrames * kHalfPad;     // [kFrames][kHalfPad]
  const int base = 16 * rev5(lane);
  const float sc = 1.0f / kM;
#pragma unroll
  for (int r = 0; r < 16; ++r) {  // x(2t) = Re / 512, x(2t+1) = -Im / 512, windowed
    const int s = 2 * (base + r);
    const float x0 = on ? __ldg(g_win + s) * u[r].x * sc : 0.f;
    const float x1 = on ? -__ldg(g_win + s + 1) * u[r].y * sc : 0.f;
    float* half = s < kH ? first + w * kHalfPad : second + w * kHalfPad;
    const int sh = s < kH ? s : s - kH;
    half[spad(sh)] = x0;
    half[spad(sh + 1)] = x1;
  }
  __syncthreads();
  // samples k H + u: second half of frame k - 1 (local k - k0) + first half of frame k (local k - k0 + 1)
  float* oc = out + (size_t)c * ((size_t)N + 1) * kH;
  const int nk = min(kFrames - 1, N + 1 - k0);
  for (int t = threadIdx.x; t < nk * kH; t += kThreads) {
    const int kk = t / kH, uu = t % kH;
    oc[(size_t)(k0 + kk) * kH + uu] = second[kk * kHalfPad + spad(uu)] + first[(kk + 1) * kHalfPad + spad(uu)];
  }
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
  if (ld < N || (ld % 4) != 0 || !x || !out || (reinterpret_cast<uintptr_t>(out) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(x) % 4) != 0 || C > 65535)
    return FFCA_ERR_ARG;
  ffca_status st = ensure_tables();
  if (st != FFCA_OK) return st;
  const size_t smem = sizeof(StftSmem);
  if (cudaFuncSetAttribute(k_stft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FFCA_ERR_CUDA;
  const dim3 grid((N + kFrames - 1) / kFrames, C);
  k_stft<<<grid, kThreads, smem, as_stream(stream)>>>(x, S, N, static_cast<float2*>(out), ld);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

ffca_status ffca_istft(const void* in, int C, int N, int ld, float* out, void* stream) {
  if (C < 0 || N < 0 || ld < 0) return FFCA_ERR_ARG;
  if (C == 0 || N == 0) return FFCA_OK;
  if (ld < N || !in || !out || (reinterpret_cast<uintptr_t>(in) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(out) % 4) != 0 || C > 65535 || N > (1 << 30) - 2)
    return FFCA_ERR_ARG;
  ffca_status st = ensure_tables();
  if (st != FFCA_OK) return st;
  const size_t smem = sizeof(StftSmem);
  if (cudaFuncSetAttribute(k_istft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FFCA_ERR_CUDA;
  const dim3 grid((N + 1 + kFrames - 2) / (kFrames - 1), C);
  k_istft<<<grid, kThreads, smem, as_stream(stream)>>>(static_cast<const float2*>(in), N, ld, out);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

}  // extern "C"
