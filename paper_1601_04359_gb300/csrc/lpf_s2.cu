// Two-point probability function of a periodic image (Sec. 2.1), the
// baseline descriptor the paper compares the lineal path function with:
//   S2_p(x, y) = 1/(W H) * IDFT( DFT(chi_p) * conj(DFT(chi_p)) )(x, y)
// with chi_p the indicator of phase p and IDFT normalised by 1/(W H); this
// equals the direct autocorrelation sum of Eq. (S2dis).  The transforms are
// cuFFT's double-precision real-to-complex / complex-to-real FFTs (a plain
// library FFT, as in the paper); the indicator, the power spectrum and the
// scaling are this library's kernels.  Plans and the spectrum buffer are
// cached per device and image size.
#include <cufft.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_state.hpp"

namespace lpf {

__global__ void s2_indicator_kernel(const uint8_t* __restrict__ img, int64_t n, int phase, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (img[i] != 0) == (phase != 0) ? 1.0 : 0.0;
}

// X <- |X|^2 (imaginary part 0), in place.
__global__ void s2_power_kernel(cufftDoubleComplex* __restrict__ X, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cufftDoubleComplex z = X[i];
    X[i] = make_cuDoubleComplex(z.x * z.x + z.y * z.y, 0.0);
  }
}

// s2 = x * scale, double -> float.
__global__ void s2_scale_kernel(const double* __restrict__ x, int64_t n, double scale, float* __restrict__ s2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s2[i] = (float)(x[i] * scale);
}

namespace {
struct S2Plan {
  int dev = -1, H = 0, W = 0;
  cufftHandle fwd = 0, inv = 0;
  double* x = nullptr;                 // [H][W]
  cufftDoubleComplex* X = nullptr;     // [H][W/2+1]
};
std::mutex g_s2_mu;
std::vector<S2Plan> g_s2_plans;

int s2_plan(int dev, int H, int W, S2Plan*& out) {
  for (S2Plan& p : g_s2_plans)
    if (p.dev == dev && p.H == H && p.W == W) { out = &p; return LPF_OK; }
  S2Plan p;
  p.dev = dev;
  p.H = H;
  p.W = W;
  // a single row or column is a 1-D transform of the other extent
  const int n1 = H == 1 ? W : H;
  const bool one_d = H == 1 || W == 1;
  if (one_d) {
    if (cufftPlan1d(&p.fwd, n1, CUFFT_D2Z, 1) != CUFFT_SUCCESS) return LPF_ECUDA;
    if (cufftPlan1d(&p.inv, n1, CUFFT_Z2D, 1) != CUFFT_SUCCESS) { cufftDestroy(p.fwd); return LPF_ECUDA; }
  } else {
    if (cufftPlan2d(&p.fwd, H, W, CUFFT_D2Z) != CUFFT_SUCCESS) return LPF_ECUDA;
    if (cufftPlan2d(&p.inv, H, W, CUFFT_Z2D) != CUFFT_SUCCESS) { cufftDestroy(p.fwd); return LPF_ECUDA; }
  }
  cudaError_t e = cudaMalloc(&p.x, sizeof(double) * (size_t)H * W);
  if (e == cudaSuccess) e = cudaMalloc(&p.X, sizeof(cufftDoubleComplex) * (size_t)(one_d ? n1 / 2 + 1 : H * (W / 2 + 1)));
  if (e != cudaSuccess) {
    cufftDestroy(p.fwd);
    cufftDestroy(p.inv);
    cudaFree(p.x);
    return set_cuda_error(e);
  }
  g_s2_plans.push_back(p);
  out = &g_s2_plans.back();
  return LPF_OK;
}
}  // namespace

}  // namespace lpf

extern "C" int s2_fft(const uint8_t* img_dev, int32_t H, int32_t W, int32_t phase, float* s2_dev,
                      lpf_stream_t stream) {
  if (!img_dev || !s2_dev || H < 1 || W < 1 || (int64_t)H * W > (1 << 26) || (phase != 0 && phase != 1))
    return LPF_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  std::lock_guard<std::mutex> lock(lpf::g_s2_mu);
  lpf::S2Plan* p = nullptr;
  int rc = (H == 1 && W == 1) ? LPF_OK : lpf::s2_plan(dev, H, W, p);
  if (rc) return rc;
  static double* one = nullptr;  // scratch for the 1x1 image
  if (H == 1 && W == 1) {
    if (!one && (e = cudaMalloc(&one, sizeof(double))) != cudaSuccess) return lpf::set_cuda_error(e);
    static lpf::S2Plan single;
    single.x = one;
    p = &single;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (H == 1 && W == 1) {  // S2(0) = chi
    (void)cudaGetLastError();
    lpf::s2_indicator_kernel<<<1, 32, 0, s>>>(img_dev, 1, phase, p->x);
    lpf::s2_scale_kernel<<<1, 32, 0, s>>>(p->x, 1, 1.0, s2_dev);
    return lpf::set_cuda_error(cudaGetLastError());
  }
  if (cufftSetStream(p->fwd, s) != CUFFT_SUCCESS || cufftSetStream(p->inv, s) != CUFFT_SUCCESS) return LPF_ECUDA;
  const int64_t n = (int64_t)H * W;
  const int64_t nc = (H == 1 || W == 1) ? n / 2 + 1 : (int64_t)H * (W / 2 + 1);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  (void)cudaGetLastError();
  lpf::s2_indicator_kernel<<<blocks, 256, 0, s>>>(img_dev, n, phase, p->x);
  if (cufftExecD2Z(p->fwd, p->x, p->X) != CUFFT_SUCCESS) return LPF_ECUDA;
  lpf::s2_power_kernel<<<(int)std::min<int64_t>((nc + 255) / 256, 4096), 256, 0, s>>>(p->X, nc);
  if (cufftExecZ2D(p->inv, p->X, p->x) != CUFFT_SUCCESS) return LPF_ECUDA;
  // cuFFT's inverse is unnormalised: IDFT = Z2D / (W H); S2 = IDFT / (W H).
  const double scale = 1.0 / ((double)n * (double)n);
  lpf::s2_scale_kernel<<<blocks, 256, 0, s>>>(p->x, n, scale, s2_dev);
  return lpf::set_cuda_error(cudaGetLastError());
}
