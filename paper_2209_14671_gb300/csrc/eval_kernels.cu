// Evaluation of Sec. 4.1 on the GPU: the degradations of Eqs. 2 and 20 applied to simulated
// intensities, the noise level NL of Eq. 21 and the LSNR of Eq. 22.
//
// Random fields (the zeta of the uneven illumination, the Gaussian noise xi, the uniforms of
// the salt & pepper rule) are inputs: the caller draws them, so results are reproducible and
// comparable with any other implementation given the same fields.
//
//   degrade:  blur rows, blur columns (circular, separable periodic Gaussian of 1/e^2 radius w),
//             then one block per image: min / max of the blurred field, and per pixel
//             I = ((1 - c) + c N(blur)) I_clean + Omega + a xi, then salt & pepper.
//   NL:       one block per image: sum |I_sim - I_noised| and sum |I_sim| (pair-of-floats sums),
//             ratios averaged over the dark-field images on the host in image order.
//   LSNR:     two passes in FP64: sums of d = truth - rec and of truth^2, then sum (d - b)^2
//             with b = mean(d), each as fixed-order block partials and one final block.
// These are HBM-bound elementwise passes (the blur is n MACs per pixel and pass).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/elfpie.h"
#include "internal.cuh"
#include "reduce.cuh"

namespace elf {
int handle_get_object_async(elf_handle h, float* obj);
cudaStream_t handle_stream(elf_handle h);
int handle_set_error(int code, const char* msg);
int handle_image_info(elf_handle h, int* n, int* N, int* n_img);
int handle_darkfield(elf_handle h, std::vector<unsigned char>& dark);
}  // namespace elf

namespace elf {
namespace {

constexpr int kBlurMax = 1024;  // longest image side the blur handles (one row in shared memory)

// fixed-order FP64 sum over a block of 256 threads; valid in thread 0; red holds 8 doubles
__device__ double block_sum_d(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();  // red may still be read by a previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// 1D periodic Gaussian exp(-2 d^2 / w^2), d the wrapped distance, normalised to unit sum;
// the 2D kernel of Eq. 20 is the product of two of these (A19, A20)
__device__ void periodic_gauss(float* g, int n, float w, float* red) {
  for (int d = threadIdx.x; d < n; d += blockDim.x) {
    const float dd = (float)min(d, n - d);
    g[d] = expf(-2.f * dd * dd / (w * w));
  }
  __syncthreads();
  float s = 0.f;
  for (int d = threadIdx.x; d < n; d += blockDim.x) s += g[d];
  const float part[1] = {s};
  double sum[1];
  block_sum_ff<1>(part, red, sum);
  __shared__ float inv;
  if (threadIdx.x == 0) inv = (float)(1.0 / sum[0]);
  __syncthreads();
  for (int d = threadIdx.x; d < n; d += blockDim.x) g[d] *= inv;
  __syncthreads();
}

// out[line][x] = sum_d g[d] in[line][(x - d) mod n] along rows (stride 1) or columns (stride n);
// one block per line; in and out may be the same array (the line is staged first)
__global__ void __launch_bounds__(256) blur_lines_kernel(const float* in, float* out, int n, float w,
                                                         int columns) {
  __shared__ float g[kBlurMax];
  __shared__ float line[kBlurMax];
  __shared__ float red[2 * 8];
  periodic_gauss(g, n, w, red);
  const size_t B = (size_t)n * n;
  const int img = blockIdx.x / n, l = blockIdx.x - img * n;
  const size_t base = img * B + (columns ? (size_t)l : (size_t)l * n);
  const size_t step = columns ? (size_t)n : 1;
  for (int x = threadIdx.x; x < n; x += blockDim.x) line[x] = in[base + x * step];
  __syncthreads();
  for (int x = threadIdx.x; x < n; x += blockDim.x) {
    float acc = 0.f;
    for (int d = 0; d < n; ++d) {
      int xs = x - d;
      xs += (xs < 0) ? n : 0;
      acc = fmaf(g[d], line[xs], acc);
    }
    out[base + x * step] = acc;
  }
}

// one block per image: illumination pattern from the blurred field held in I_out (if c != 0),
// then background, Gaussian noise and salt & pepper; every pixel is read and written by the
// same thread after the block's min / max
__global__ void __launch_bounds__(1024) compose_kernel(const float* __restrict__ I_clean, float* I_out,
                                                       const float* __restrict__ background,
                                                       const float* __restrict__ xi,
                                                       const float* __restrict__ u_snp, int n, float c,
                                                       float a, double snp) {
  __shared__ float rmin[32], rmax[32];
  __shared__ float lo_s, span_s;
  const size_t B = (size_t)n * n;
  const size_t base = blockIdx.x * B;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (c != 0.f) {
    float lo = INFINITY, hi = -INFINITY;
    for (size_t p = t; p < B; p += blockDim.x) {
      const float v = I_out[base + p];
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
    for (int off = 16; off > 0; off >>= 1) {
      lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, off));
      hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) {
      rmin[wid] = lo;
      rmax[wid] = hi;
    }
    __syncthreads();
    if (t == 0) {
      float l = rmin[0], h = rmax[0];
      for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
        l = fminf(l, rmin[i]);
        h = fmaxf(h, rmax[i]);
      }
      lo_s = l;
      span_s = h - l;
    }
    __syncthreads();
  }
  const float lo = (c != 0.f) ? lo_s : 0.f, span = (c != 0.f) ? span_s : 0.f;
  const float bg = background ? background[blockIdx.x] : 0.f;
  for (size_t p = t; p < B; p += blockDim.x) {
    float v = I_clean[base + p];
    if (c != 0.f) {
      const float nrm = (span > 0.f) ? (I_out[base + p] - lo) / span : 0.f;
      v *= (1.f - c) + c * nrm;
    }
    v += bg;
    if (a != 0.f) v = fmaf(a, xi[base + p], v);
    if (snp != 0.0) {
      const float u = u_snp[base + p];
      // the thresholds in FP64, as the density is given, so the decisions match an FP64 evaluation
      v = ((double)u < 0.5 * snp) ? 0.f : ((double)u < snp) ? 1.f : v;
    }
    I_out[base + p] = v;
  }
}

// one block per image: sum |a - b| and sum |a| (Eq. 21), FP64-accurate pair sums
__global__ void __launch_bounds__(1024) l1_ratio_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                        size_t B, double* out2) {
  __shared__ float red[2 * 2 * 32];
  const size_t base = blockIdx.x * B;
  FF s[2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (size_t p = threadIdx.x; p < B; p += blockDim.x) {
    const float x = a[base + p], y = b[base + p];
    s[0] = ff_add(s[0], FF{fabsf(x - y), 0.f});
    s[1] = ff_add(s[1], FF{fabsf(x), 0.f});
  }
  double sum[2];
  block_sum_ff<2>(s, red, sum);
  if (threadIdx.x == 0) {
    out2[2 * blockIdx.x] = sum[0];
    out2[2 * blockIdx.x + 1] = sum[1];
  }
}

constexpr int kLsnrBlocks = 1024;  // partials of each LSNR pass (grid-stride blocks)

// pass 1: partial sums of d = truth - rec and of truth^2 in FP64; values are x[i * stride]
__global__ void __launch_bounds__(256) lsnr_pass1_kernel(const float* __restrict__ rec,
                                                         const float* __restrict__ truth, size_t count, int stride,
                                                         double* part) {
  __shared__ double red[8];
  double sd = 0.0, st = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double t = truth[i * stride], r = rec[i * stride];
    sd += t - r;
    st += t * t;
  }
  const double a = block_sum_d(sd, red);
  const double b = block_sum_d(st, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// pass 2: partial sums of (d - b)^2 with b = sum d / count taken from pass 1's partials
__global__ void __launch_bounds__(256) lsnr_pass2_kernel(const float* __restrict__ rec,
                                                         const float* __restrict__ truth, size_t count, int stride,
                                                         const double* part1, double* part2) {
  __shared__ double red[8];
  __shared__ double b_s;
  if (threadIdx.x == 0) {
    double sd = 0.0;
    for (int i = 0; i < kLsnrBlocks; ++i) sd += part1[2 * i];
    b_s = sd / (double)count;
  }
  __syncthreads();
  const double b = b_s;
  double se = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double e = ((double)truth[i * stride] - (double)rec[i * stride]) - b;
    se += e * e;
  }
  const double a = block_sum_d(se, red);
  if (threadIdx.x == 0) part2[blockIdx.x] = a;
}

// object quality: the least-squares global phase sum conj(rec) truth (pair sums per block)
__global__ void __launch_bounds__(256) phase_dot_kernel(const float2* __restrict__ rec,
                                                        const float2* __restrict__ truth, size_t count,
                                                        double* part) {
  __shared__ float red[2 * 2 * 8];
  FF s[2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 r = rec[i], t = truth[i];
    s[0] = ff_add(s[0], FF{r.x * t.x + r.y * t.y, 0.f});
    s[1] = ff_add(s[1], FF{r.x * t.y - r.y * t.x, 0.f});
  }
  double sum[2];
  block_sum_ff<2>(s, red, sum);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sum[0];
    part[2 * blockIdx.x + 1] = sum[1];
  }
}

// amplitude and phase of rec e^{i phi0} and of truth, as (amplitude, phase) pairs
__global__ void __launch_bounds__(256) amp_phase_kernel(const float2* __restrict__ rec,
                                                        const float2* __restrict__ truth, size_t count, float c0,
                                                        float s0, float2* ap_rec, float2* ap_true) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 r = rec[i], t = truth[i];
    const float ax = r.x * c0 - r.y * s0, ay = r.x * s0 + r.y * c0;
    ap_rec[i] = make_float2(sqrtf(ax * ax + ay * ay), atan2f(ay, ax));
    ap_true[i] = make_float2(sqrtf(t.x * t.x + t.y * t.y), atan2f(t.y, t.x));
  }
}

}  // namespace
}  // namespace elf

// ------------------------------------------------------------------ C ABI
namespace {

int cuda_fail(cudaError_t e, const char* where) {
  return elf::handle_set_error(ELF_ECUDA, (std::string(where) + ": " + cudaGetErrorString(e)).c_str());
}

// LSNR of Eq. 22 from x[i * stride], i < count, device arrays; synchronises s
int lsnr_impl(const float* rec, const float* truth, size_t count, int stride, cudaStream_t s, double* out) {
  double* part = nullptr;
  cudaError_t e = cudaMalloc(&part, sizeof(double) * 3 * elf::kLsnrBlocks);
  if (e != cudaSuccess) return elf::handle_set_error(ELF_ENOMEM, "elf_lsnr: scratch allocation failed");
  elf::lsnr_pass1_kernel<<<elf::kLsnrBlocks, 256, 0, s>>>(rec, truth, count, stride, part);
  elf::lsnr_pass2_kernel<<<elf::kLsnrBlocks, 256, 0, s>>>(rec, truth, count, stride, part,
                                                          part + 2 * elf::kLsnrBlocks);
  std::vector<double> h(3 * elf::kLsnrBlocks);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "elf_lsnr");
  double tt = 0.0, ee = 0.0;
  for (int i = 0; i < elf::kLsnrBlocks; ++i) {
    tt += h[2 * i + 1];
    ee += h[2 * elf::kLsnrBlocks + i];
  }
  *out = 10.0 * std::log10(tt / ee);
  return ELF_OK;
}

}  // namespace

extern "C" int elf_lsnr(const float* rec, const float* truth, long long count, void* cuda_stream, double* out) {
  if (!rec || !truth || !out || count < 1) return elf::handle_set_error(ELF_EINVAL, "elf_lsnr: bad arguments");
  return lsnr_impl(rec, truth, (size_t)count, 1, static_cast<cudaStream_t>(cuda_stream), out);
}

extern "C" int elf_degrade(elf_handle h, const float* I_clean, const float* zeta, const float* background,
                           const float* xi, const float* u_snp, const elf_degrade_params* prm, float* I_out) {
  if (!h || !I_clean || !I_out || !prm) return elf::handle_set_error(ELF_EINVAL, "elf_degrade: null argument");
  const double c = prm->illum_c, w = prm->waist_px, a = prm->gauss_a, d = prm->snp_density;
  if (!(std::isfinite(c) && c >= 0 && c <= 1 && std::isfinite(a) && std::isfinite(d) && d >= 0 && d <= 1))
    return elf::handle_set_error(ELF_EINVAL, "elf_degrade: need 0 <= illum_c <= 1, finite gauss_a, 0 <= density <= 1");
  if ((c != 0 && (!zeta || !(w > 0 && std::isfinite(w)))) || (a != 0 && !xi) || (d != 0 && !u_snp))
    return elf::handle_set_error(ELF_EINVAL, "elf_degrade: a random field or the waist is missing");
  if (I_out == I_clean || I_out == zeta || I_out == xi || I_out == u_snp)
    return elf::handle_set_error(ELF_EINVAL, "elf_degrade: I_out must not alias an input");
  int n = 0, N = 0, n_img = 0;
  elf::handle_image_info(h, &n, &N, &n_img);
  if (n > elf::kBlurMax) return elf::handle_set_error(ELF_EINVAL, "elf_degrade: image side too large");
  cudaStream_t s = elf::handle_stream(h);
  if (c != 0) {
    elf::blur_lines_kernel<<<n_img * n, 256, 0, s>>>(zeta, I_out, n, (float)w, 0);
    elf::blur_lines_kernel<<<n_img * n, 256, 0, s>>>(I_out, I_out, n, (float)w, 1);
  }
  elf::compose_kernel<<<n_img, 1024, 0, s>>>(I_clean, I_out, background, xi, u_snp, n, (float)c, (float)a, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? ELF_OK : cuda_fail(e, "elf_degrade");
}

extern "C" int elf_noise_level(elf_handle h, const float* I_sim, const float* I_noised, double* nl) {
  if (!h || !I_sim || !I_noised || !nl) return elf::handle_set_error(ELF_EINVAL, "elf_noise_level: null argument");
  int n = 0, N = 0, n_img = 0;
  elf::handle_image_info(h, &n, &N, &n_img);
  std::vector<unsigned char> dark;
  elf::handle_darkfield(h, dark);
  cudaStream_t s = elf::handle_stream(h);
  double* part = nullptr;
  if (cudaMalloc(&part, sizeof(double) * 2 * n_img) != cudaSuccess)
    return elf::handle_set_error(ELF_ENOMEM, "elf_noise_level: scratch allocation failed");
  elf::l1_ratio_kernel<<<n_img, 1024, 0, s>>>(I_sim, I_noised, (size_t)n * n, part);
  std::vector<double> hp(2 * (size_t)n_img);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "elf_noise_level");
  double acc = 0.0;
  int cnt = 0;
  for (int j = 0; j < n_img; ++j)
    if (dark[j]) {
      acc += hp[2 * j] / hp[2 * j + 1];
      ++cnt;
    }
  *nl = cnt ? 100.0 * acc / cnt : 0.0;
  return ELF_OK;
}

extern "C" int elf_object_quality(elf_handle h, const float* obj_true, double* out2) {
  if (!h || !obj_true || !out2) return elf::handle_set_error(ELF_EINVAL, "elf_object_quality: null argument");
  int n = 0, N = 0, n_img = 0;
  elf::handle_image_info(h, &n, &N, &n_img);
  const size_t A = (size_t)N * N;
  cudaStream_t s = elf::handle_stream(h);
  float2* buf = nullptr;  // the reconstructed object, then (amplitude, phase) of it and of the truth
  if (cudaMalloc(&buf, sizeof(float2) * 3 * A) != cudaSuccess)
    return elf::handle_set_error(ELF_ENOMEM, "elf_object_quality: scratch allocation failed");
  double* part = nullptr;
  if (cudaMalloc(&part, sizeof(double) * 2 * elf::kLsnrBlocks) != cudaSuccess) {
    cudaFree(buf);
    return elf::handle_set_error(ELF_ENOMEM, "elf_object_quality: scratch allocation failed");
  }
  int rc = elf::handle_get_object_async(h, reinterpret_cast<float*>(buf));
  const float2* truth = reinterpret_cast<const float2*>(obj_true);
  std::vector<double> hp(2 * elf::kLsnrBlocks);
  cudaError_t e = cudaSuccess;
  if (rc == ELF_OK) {
    elf::phase_dot_kernel<<<elf::kLsnrBlocks, 256, 0, s>>>(buf, truth, A, part);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (rc == ELF_OK && e == cudaSuccess) {
    double re = 0.0, im = 0.0;
    for (int i = 0; i < elf::kLsnrBlocks; ++i) {
      re += hp[2 * i];
      im += hp[2 * i + 1];
    }
    const double phi0 = std::atan2(im, re);
    elf::amp_phase_kernel<<<elf::kLsnrBlocks, 256, 0, s>>>(buf, truth, A, (float)std::cos(phi0),
                                                           (float)std::sin(phi0), buf + A, buf + 2 * A);
    e = cudaGetLastError();
    const float* rec_ap = reinterpret_cast<const float*>(buf + A);
    const float* true_ap = reinterpret_cast<const float*>(buf + 2 * A);
    if (e == cudaSuccess) rc = lsnr_impl(rec_ap, true_ap, A, 2, s, &out2[0]);
    if (e == cudaSuccess && rc == ELF_OK) rc = lsnr_impl(rec_ap + 1, true_ap + 1, A, 2, s, &out2[1]);
  }
  cudaFree(part);
  cudaFree(buf);
  if (rc != ELF_OK) return rc;
  return e == cudaSuccess ? ELF_OK : cuda_fail(e, "elf_object_quality");
}
