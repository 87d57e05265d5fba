// STFT front end and inverse (overlap-add) back end with the parameters of
// the paper's experiments (Table 1: frame length L = 1024, shift H = 512,
// square root of the Hann window; bins up to the Nyquist frequency, F = 513,
// Sec. 2).  The frame's 1024 real samples are transformed as one 512-point
// complex FFT of z(t) = x(2t) + i x(2t+1) (radix-8 Stockham, three stages in
// shared memory, 64 threads per transform), then split into the spectrum of
// the real frame:
//     X[k] = E[k] + e^{-2 pi i k/1024} O[k],  E[k] = (Z[k] + conj Z[512-k]) / 2,
//     O[k] = (Z[k] - conj Z[512-k]) / (2i),   k = 0 .. 512 (Z[512] = Z[0]).
// The inverse runs the same steps backwards.  FP32 data, twiddles and window
// rounded from FP64 values computed on the host.
//
// A CTA takes kFrames consecutive frames of one channel: the overlapping
// samples are read once, and the spectra leave as runs of kFrames
// consecutive frames of one bin (the frame-contiguous mic-planar layout).
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
constexpr int kFrames = 8;      // frames per CTA
constexpr int kThreads = 256;   // four 64-thread transform groups
constexpr int kGroups = kThreads / 64;
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

// 8-point DFT in registers: two 4-point DFTs of the even and odd entries,
// joined with the twiddles e^{-2 pi i q / 8}.
__device__ inline void dft8(float2 (&u)[8]) {
  float2 e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
  float2 o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const float r = 0.70710678118654752f;
  o1 = make_float2(r * (o1.x + o1.y), r * (o1.y - o1.x));    // * (1 - i) / sqrt 2
  o2 = mul_mi(o2);                                           // * (-i)
  o3 = make_float2(r * (o3.y - o3.x), -r * (o3.x + o3.y));   // * (-1 - i) / sqrt 2
  u[0] = cadd(e0, o0);
  u[4] = csub(e0, o0);
  u[1] = cadd(e1, o1);
  u[5] = csub(e1, o1);
  u[2] = cadd(e2, o2);
  u[6] = csub(e2, o2);
  u[3] = cadd(e3, o3);
  u[7] = csub(e3, o3);
}

// Forward 512-point DFT of a[0..511] by one 64-thread group (thread j):
// three radix-8 Stockham stages a -> b -> a -> b (result in b).  At stage p
// (sub-transform size p = 1, 8, 64) thread j takes u_r = src[j + 64 r],
// twiddles u_r by e^{-2 pi i r k / (8 p)} (k = j mod p), transforms, and
// writes dst[(j - k) 8 + k + p r].  group_sync() separates the stages.
template <typename Sync>
__device__ void fft512(float2* a, float2* b, const float2* tw, int j, Sync group_sync) {
  float2* src = a;
  float2* dst = b;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = s == 0 ? 1 : (s == 1 ? 8 : 64);
    const int k = j & (p - 1);
    float2 u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) u[r] = src[j + 64 * r];
    if (s > 0) {
#pragma unroll
      for (int r = 1; r < 8; ++r) u[r] = cmul(u[r], tw[(r * k * (64 / p)) & (kM - 1)]);
    }
    dft8(u);
    const int base = (j - k) * 8 + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) dst[base + p * r] = u[r];
    group_sync();
    float2* t = src;
    src = dst;
    dst = t;
  }
}

// Shared memory of one CTA (floats/float2 arrays carved from one buffer).
struct StftSmem {
  float2 tw512[kM];
  float2 tw1024[kF + 3];
  float win[kL];
  float2 fft[kGroups][2][kM];
  float2 spec[kF][kFrames];   // the CTA's spectra, bin-major
  float samp[(kFrames + 1) * kH];
};

template <typename Smem>
__device__ inline void load_tables(Smem& sm) {
  for (int t = threadIdx.x; t < kM; t += kThreads) sm.tw512[t] = g_tw512[t];
  for (int t = threadIdx.x; t < kF; t += kThreads) sm.tw1024[t] = g_tw1024[t];
  for (int t = threadIdx.x; t < kL; t += kThreads) sm.win[t] = g_win[t];
}

// x [C][S] float -> out [C][F][ld] complex64 (frames 0 .. N-1, then zero to ld).
__global__ void __launch_bounds__(kThreads) k_stft(const float* __restrict__ x, long long S, int N,
                                                   float2* __restrict__ out, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftSmem& sm = *reinterpret_cast<StftSmem*>(smem_raw);
  const int c = blockIdx.y;
  const int n0 = blockIdx.x * kFrames;
  const int nf = min(kFrames, N - n0);
  const float* xc = x + (size_t)c * S;
  load_tables(sm);
  // samples n0 H .. (n0 + nf - 1) H + L - 1, all inside the signal
  const int ns = (nf + 1) * kH;
  for (int t = threadIdx.x; t < ns; t += kThreads) sm.samp[t] = __ldg(xc + (size_t)n0 * kH + t);
  __syncthreads();
  const int grp = threadIdx.x / 64, j = threadIdx.x % 64;
  auto sync = [] { __syncthreads(); };
  for (int fb = 0; fb < kFrames; fb += kGroups) {  // every thread runs every round (barriers)
    const int fr = fb + grp;
    const bool on = fr < nf;
    float2* A = sm.fft[grp][0];
    float2* B = sm.fft[grp][1];
    for (int t = j; t < kM; t += 64) {
      const int s0 = fr * kH + 2 * t;
      A[t] = on ? make_float2(sm.win[2 * t] * sm.samp[s0], sm.win[2 * t + 1] * sm.samp[s0 + 1])
                : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft512(A, B, sm.tw512, j, sync);  // Z in B
    for (int k = j; k < kF; k += 64) {
      const float2 zk = B[k & (kM - 1)];
      const float2 zm = cconj(B[(kM - k) & (kM - 1)]);
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
      const float2 o = mul_mi(make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y - zm.y)));
      if (on) sm.spec[k][fr] = cadd(e, cmul(sm.tw1024[k], o));
    }
    __syncthreads();
  }
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

// in [C][F][ld] complex64 (frames 0 .. N-1) -> out [C][(N + 1) H] float: the
// CTA writes samples k H .. k H + H - 1 for k = k0 .. k0 + kFrames - 1 (k <=
// N), each the second half of frame k - 1 plus the first half of frame k
// (windowed inverse DFTs; a missing frame adds nothing).
__global__ void __launch_bounds__(kThreads) k_istft(const float2* __restrict__ in, int N, int ld,
                                                    float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StftSmem& sm = *reinterpret_cast<StftSmem*>(smem_raw);
  // the windowed halves of frames m0 .. m0 + kFrames: first halves in samp[],
  // second halves in spec[] (unused by the inverse otherwise).  Staging the
  // spectra in shared memory for coalesced loads needs another 37 KB, which
  // halves the resident CTAs and measured slower (0.91 against 0.58 ms for
  // nine channels of 20000 frames).
  static_assert(sizeof(StftSmem::spec) / sizeof(float) >= (kFrames + 1) * kH, "second halves fit");
  static_assert(sizeof(StftSmem::samp) / sizeof(float) >= (kFrames + 1) * kH, "first halves fit");
  const int c = blockIdx.y;
  const int k0 = blockIdx.x * kFrames;
  const int m0 = k0 - 1;  // frames m0 .. m0 + kFrames
  const float2* ic = in + (size_t)c * kF * ld;
  float* first = sm.samp;                              // [kFrames + 1][H]
  float* second = reinterpret_cast<float*>(sm.spec);   // [kFrames + 1][H]
  load_tables(sm);
  __syncthreads();
  const int grp = threadIdx.x / 64, j = threadIdx.x % 64;
  auto sync = [] { __syncthreads(); };
  for (int fb = 0; fb < kFrames + 1; fb += kGroups) {
    const int fr = fb + grp;  // local frame index 0 .. kFrames
    const int m = m0 + fr;
    const bool on = fr <= kFrames && m >= 0 && m < N;
    float2* A = sm.fft[grp][0];
    float2* B = sm.fft[grp][1];
    // Z[k] = E[k] + i O[k] from X[k] and X[512 - k], conjugated for the
    // forward transform (IDFT(Z) = conj(DFT(conj Z)) / 512)
    for (int k = j; k < kM; k += 64) {
      float2 z = make_float2(0.f, 0.f);
      if (on) {
        float2 xk = __ldg(ic + (size_t)k * ld + m);
        float2 xm = cconj(__ldg(ic + (size_t)(kM - k) * ld + m));
        if (k == 0) {  // bins 0 and L/2 of a real signal's spectrum are real: their imaginary parts are ignored
          xk.y = 0.f;
          xm.y = 0.f;
        }
        const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y + xm.y));
        const float2 o = cmul(make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y - xm.y)), cconj(sm.tw1024[k]));
        z = cconj(make_float2(e.x - o.y, e.y + o.x));  // conj(E + i O)
      }
      A[k] = z;
    }
    __syncthreads();
    fft512(A, B, sm.tw512, j, sync);  // DFT(conj Z) in B
    if (fr <= kFrames) {
      const float sc = 1.0f / kM;
      for (int t = j; t < kM; t += 64) {
        const float2 zt = B[t];  // z(t) = conj(zt) / 512: x(2t) = Re, x(2t+1) = Im
        const float x0 = zt.x * sc, x1 = -zt.y * sc;
        const int s = 2 * t;
        float* dst = s < kH ? first + fr * kH + s : second + fr * kH + (s - kH);
        dst[0] = on ? sm.win[s] * x0 : 0.f;
        dst[1] = on ? sm.win[s + 1] * x1 : 0.f;
      }
    }
    __syncthreads();
  }
  // samples k H + u: second half of frame k - 1 (local k - k0) + first half of frame k (local k - k0 + 1)
  float* oc = out + (size_t)c * ((size_t)N + 1) * kH;
  const int nk = min(kFrames, N + 1 - k0);
  for (int t = threadIdx.x; t < nk * kH; t += kThreads) {
    const int kk = t / kH, u = t % kH;
    oc[(size_t)(k0 + kk) * kH + u] = second[kk * kH + u] + first[(kk + 1) * kH + u];
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
  const dim3 grid((N + 1 + kFrames - 1) / kFrames, C);
  k_istft<<<grid, kThreads, smem, as_stream(stream)>>>(static_cast<const float2*>(in), N, ld, out);
  return cudaGetLastError() == cudaSuccess ? FFCA_OK : FFCA_ERR_CUDA;
}

}  // extern "C"
