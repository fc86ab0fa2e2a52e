// Multiplexed illumination (Eq. 1 with M > 1 LEDs per measured image).
//
// Image j is lit by LEDs jM .. jM+M-1 and its model intensity is s_j = sum_m |o_{j,m}|^2,
// so the residual, its gradient, the normaliser and the divergence of Eqs. 5 (4), 12 and
// 11 (10) are per image, shared by the image's M LEDs:
//
//   f_j = g'(s_j) * nabla^T omega(nabla r_j),   r_j = g(s_j) - g(max(I_j, 0)),
//
// and each LED's tile only needs W_{j,m} = o_{j,m} * f_j (the tile kernel's mode 2).
// The iteration's tile stage for M > 1 is therefore
//   1. tile kernel, mode 1: |o_k|^2 for every LED k (K x n x n);
//   2. mux_resid_kernel: s_j in ascending m, r_j and the slope g'(s_j) (K/M x n x n);
//   3. mux_omega_kernel: nabla, omega (Huber smoothing, isotropic or not), nabla^T, f_j,
//      and the fidelity cost of every image, as FP64-accurate partials per block;
//   4. tile kernel, mode 2: W = o * f_j, forward transform, G on the support.
// Everything here is elementwise or a 3-point stencil on n x n images: HBM / L2 bound.
#include <algorithm>

#include "internal.cuh"
#include "reduce.cuh"

namespace elf {

namespace {

// r and g'(s) of one pixel for the model intensity s and the measured value meas (the
// measurement itself for fidelity 0, the mapped g(max(I, 0)) for 1, 2 and 3)
__device__ __forceinline__ void resid_slope(float s, float meas, int fidelity, float gexp, float eta, float& r,
                                            float& slope) {
  if (fidelity == 0) {  // Eq. 5: r = s - I, dr/ds = 1
    r = s - meas;
    slope = 1.f;
  } else if (fidelity == 1) {  // Eq. 4: r = sqrt(s) - sqrt(max(I, 0)), g' = 1 / (2 max(sqrt(s), eta))
    const float a = sqrtf(s);
    r = a - meas;  // meas holds sqrt(max(I, 0))
    slope = 1.f / (2.f * fmaxf(a, eta));
  } else if (fidelity == 2) {  // Sec. 6.3 power map
    r = powf(s, gexp) - meas;
    slope = gexp * powf(fmaxf(s, eta * eta), gexp - 1.f);
  } else {  // Sec. 6.3 log map
    r = log1pf(s) - meas;
    slope = 1.f / (s + 1.f);
  }
}

struct Omega {
  float wx, wy, phi;
};

// Huber-smoothed L1 normaliser of Eq. 12 at one pixel: omega = d / max(|d|, tau) (isotropic)
// or componentwise (anisotropic), and the smoothed cost phi; the same arithmetic as the
// single-LED stencil of the tile kernel
__device__ __forceinline__ Omega omega_at(float dx, float dy, float tau, int iso) {
  Omega o;
  const float hit = (tau > 0.f) ? 0.5f / tau : 0.f;
  if (iso) {
    const float ss = dx * dx + dy * dy;
    const float inv = rsqrtf(fmaxf(ss, fmaxf(tau * tau, 1e-36f)));
    o.wx = dx * inv;
    o.wy = dy * inv;
    o.phi = (ss >= tau * tau) ? ss * inv : ss * hit + 0.5f * tau;
  } else {
    const float ax = fabsf(dx), ay = fabsf(dy);
    o.wx = dx / fmaxf(ax, fmaxf(tau, 1e-18f));  // 0 at the origin when tau = 0
    o.wy = dy / fmaxf(ay, fmaxf(tau, 1e-18f));
    o.phi = ((ax >= tau) ? ax : ax * ax * hit + 0.5f * tau) + ((ay >= tau) ? ay : ay * ay * hit + 0.5f * tau);
  }
  return o;
}

// s_j = sum over the image's LEDs in ascending order, r_j and g'(s_j); four pixels per thread
__global__ void __launch_bounds__(256) mux_resid_kernel(const float4* __restrict__ Imod,
                                                        const float4* __restrict__ meas, float4* __restrict__ R,
                                                        float4* __restrict__ F, int n_img, int M, int B4,
                                                        int fidelity, float gexp, float eta) {
  const size_t total = (size_t)n_img * B4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = i / B4, p = i - j * B4;
    float4 s = Imod[(j * M) * B4 + p];
    for (int m = 1; m < M; ++m) {
      const float4 v = Imod[(j * M + m) * B4 + p];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    const float4 q = meas[i];
    float4 r, f;
    resid_slope(s.x, q.x, fidelity, gexp, eta, r.x, f.x);
    resid_slope(s.y, q.y, fidelity, gexp, eta, r.y, f.y);
    resid_slope(s.z, q.z, fidelity, gexp, eta, r.z, f.z);
    resid_slope(s.w, q.w, fidelity, gexp, eta, r.w, f.w);
    R[i] = r;
    F[i] = f;
  }
}

// f_j = g'(s_j) nabla^T omega(nabla r_j) in place of the slope, one pixel per thread, blocks of
// 256 consecutive pixels of one image; per-block cost partials (fixed order, FP64-accurate)
__global__ void __launch_bounds__(256) mux_omega_kernel(const float* __restrict__ R, float* __restrict__ F,
                                                        double* __restrict__ partial, int n, int bpi, float tau,
                                                        int iso) {
  __shared__ float red[2 * 8];
  const int B = n * n;
  const int j = blockIdx.x / bpi, blk = blockIdx.x - j * bpi;
  const int p = blk * 256 + threadIdx.x;
  const float* r = R + (size_t)j * B;
  float phi = 0.f;
  if (p < B) {
    const int y = p / n, x = p - y * n;
    // forward differences with a zero last row / column (Neumann)
    auto rr = [&](int yy, int xx) { return __ldg(r + yy * n + xx); };
    const float r0 = rr(y, x);
    const float dx = (x < n - 1) ? rr(y, x + 1) - r0 : 0.f;
    const float dy = (y < n - 1) ? rr(y + 1, x) - r0 : 0.f;
    const Omega w0 = omega_at(dx, dy, tau, iso);
    phi = w0.phi;
    float w = -w0.wx - w0.wy;
    if (x >= 1) {  // omega_x one pixel to the left
      const float rl = rr(y, x - 1);
      const float dyl = (y < n - 1) ? rr(y + 1, x - 1) - rl : 0.f;
      w += omega_at(r0 - rl, dyl, tau, iso).wx;
    }
    if (y >= 1) {  // omega_y one pixel above
      const float ru = rr(y - 1, x);
      const float dxu = (x < n - 1) ? rr(y - 1, x + 1) - ru : 0.f;
      w += omega_at(dxu, r0 - ru, tau, iso).wy;
    }
    float* f = F + (size_t)j * B + p;
    *f = *f * w;
  }
  const float part[1] = {phi};
  double sum[1];
  block_sum_ff<1>(part, red, sum);
  if (threadIdx.x == 0) partial[blockIdx.x] = sum[0];
}

// sum over the image's LEDs (the multiplexed forward model of Eq. 1), ascending m
__global__ void __launch_bounds__(256) mux_sum_kernel(const float4* __restrict__ Imod, float4* __restrict__ out,
                                                      int n_img, int M, int B4) {
  const size_t total = (size_t)n_img * B4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = i / B4, p = i - j * B4;
    float4 s = Imod[(j * M) * B4 + p];
    for (int m = 1; m < M; ++m) {
      const float4 v = Imod[(j * M + m) * B4 + p];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    out[i] = s;
  }
}

int grid_for(size_t items) { return (int)std::min<size_t>((items + 255) / 256, 152 * 16); }

}  // namespace

int mux_blocks_per_image(int n) { return (n * n + 255) / 256; }

cudaError_t launch_mux_resid(const float* Imod, const float* meas, float* R, float* F, int n_img, int M, int n,
                             int fidelity, float gexp, float eta, cudaStream_t s) {
  const int B4 = n * n / 4;  // n >= 16: whole float4 groups; buffers from cudaMalloc are 256-byte aligned
  mux_resid_kernel<<<grid_for((size_t)n_img * B4), 256, 0, s>>>(
      reinterpret_cast<const float4*>(Imod), reinterpret_cast<const float4*>(meas), reinterpret_cast<float4*>(R),
      reinterpret_cast<float4*>(F), n_img, M, B4, fidelity, gexp, eta);
  return cudaGetLastError();
}

cudaError_t launch_mux_omega(const float* R, float* F, double* partial, int n_img, int n, float tau, int iso,
                             cudaStream_t s) {
  const int bpi = mux_blocks_per_image(n);
  mux_omega_kernel<<<n_img * bpi, 256, 0, s>>>(R, F, partial, n, bpi, tau, iso);
  return cudaGetLastError();
}

cudaError_t launch_mux_sum(const float* Imod, float* out, int n_img, int M, int n, cudaStream_t s) {
  const int B4 = n * n / 4;
  mux_sum_kernel<<<grid_for((size_t)n_img * B4), 256, 0, s>>>(reinterpret_cast<const float4*>(Imod),
                                                              reinterpret_cast<float4*>(out), n_img, M, B4);
  return cudaGetLastError();
}

}  // namespace elf
