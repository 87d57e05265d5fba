// Instantiations and launches of the mask-based initialisation kernels
// (ffca_mask.cuh) for every compiled precision and microphone count.
#include <cuda_runtime.h>

#include "ffca_dispatch.h"
#include "ffca_mask.cuh"

namespace ffca {

namespace {

template <typename T, int I>
cudaError_t launch_mask(const MaskArgs& a, int problems, cudaStream_t s) {
  const dim3 gc(problems, a.J);
  k_mask_cov<T, I><<<gc, kBlock, 0, s>>>(a);
  k_mask_ajd<I><<<(problems + 63) / 64, 64, 0, s>>>(a);
  k_mask_v<T, I><<<problems, kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mask_i(const MaskArgs& a, int problems, cudaStream_t s) {
  switch (a.I) {
    case 1: return launch_mask<T, 1>(a, problems, s);
    case 2: return launch_mask<T, 2>(a, problems, s);
    case 3: return launch_mask<T, 3>(a, problems, s);
    case 4: return launch_mask<T, 4>(a, problems, s);
    case 8: return launch_mask<T, 8>(a, problems, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_mask_init(int prec, const MaskArgs& a, int problems, cudaStream_t s) {
  return prec == 0 ? launch_mask_i<double>(a, problems, s) : launch_mask_i<float>(a, problems, s);
}

}  // namespace ffca
