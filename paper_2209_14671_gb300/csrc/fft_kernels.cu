// Two-pass 2D FFT of an L x L complex array (the F_A of Eqs. 6-7, 13-14 and
// the object <-> spectrum maps).  Pass 1 transforms rows: each team of a CTA
// loads one row with coalesced float2 loads into shared memory, transforms it and
// writes it back.  Pass 2 transforms columns: a CTA loads an L x CW strip
// (coalesced CW-wide row segments), stores it column-major with a padded pitch,
// transforms each column and writes the strip back.
#include "fft.cuh"
#include "internal.cuh"

namespace elf {

constexpr int kFftThreads = 256;

template <int L, bool INV>
__global__ void __launch_bounds__(kFftThreads) fft_rows_kernel(float2* __restrict__ data, const float2* __restrict__ twg) {
  constexpr int TL = FftTeam<L>::TL;
  constexpr int NTEAM = kFftThreads / TL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* rows = tw + L;
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += kFftThreads) tw[i] = twg[i];
  const int row0 = blockIdx.x * NTEAM;
  // coalesced load of NTEAM rows
  for (int i = tid; i < NTEAM * L; i += kFftThreads) {
    const int r = i / L, x = i - r * L;
    rows[r * L + x] = (row0 + r < L) ? data[(size_t)(row0 + r) * L + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int team = tid / TL, lane = tid % TL;
  team_fft<L, INV>(rows + team * L, tw, lane, row0 + team < L);
  __syncthreads();
  for (int i = tid; i < NTEAM * L; i += kFftThreads) {
    const int r = i / L, x = i - r * L;
    if (row0 + r < L) data[(size_t)(row0 + r) * L + x] = rows[r * L + x];
  }
}

template <int L, bool INV>
__global__ void __launch_bounds__(kFftThreads) fft_cols_kernel(float2* __restrict__ data, const float2* __restrict__ twg) {
  constexpr int TL = FftTeam<L>::TL;
  constexpr int CW = kFftThreads / TL;  // columns per CTA (one team each)
  constexpr int LD = L + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* cols = tw + L;
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += kFftThreads) tw[i] = twg[i];
  const int c0 = blockIdx.x * CW;
  for (int i = tid; i < CW * L; i += kFftThreads) {
    const int y = i / CW, c = i - y * CW;
    cols[c * LD + y] = (c0 + c < L) ? data[(size_t)y * L + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int team = tid / TL, lane = tid % TL;
  team_fft<L, INV>(cols + team * LD, tw, lane, c0 + team < L);
  __syncthreads();
  for (int i = tid; i < CW * L; i += kFftThreads) {
    const int y = i / CW, c = i - y * CW;
    if (c0 + c < L) data[(size_t)y * L + c0 + c] = cols[c * LD + y];
  }
}

template <int L, bool INV>
static cudaError_t fft2_t(float2* data, const float2* tw, cudaStream_t s) {
  constexpr int TL = FftTeam<L>::TL;
  constexpr int NTEAM = kFftThreads / TL;
  const size_t smem_r = 8 * ((size_t)L + (size_t)NTEAM * L);
  const size_t smem_c = 8 * ((size_t)L + (size_t)NTEAM * (L + 1));
  const int blocks = (L + NTEAM - 1) / NTEAM;
  fft_rows_kernel<L, INV><<<blocks, kFftThreads, smem_r, s>>>(data, tw);
  fft_cols_kernel<L, INV><<<blocks, kFftThreads, smem_c, s>>>(data, tw);
  return cudaGetLastError();
}

template <int L, bool INV>
static cudaError_t prepare_fft_t() {
  constexpr int TL = FftTeam<L>::TL;
  constexpr int NTEAM = kFftThreads / TL;
  const int smem_r = (int)(8 * ((size_t)L + (size_t)NTEAM * L));
  const int smem_c = (int)(8 * ((size_t)L + (size_t)NTEAM * (L + 1)));
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_r);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_cols_kernel<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c);
}

cudaError_t prepare_fft(int L) {
#define ELF_PREP_CASE(LL)                                   \
  case LL: {                                                \
    cudaError_t e = prepare_fft_t<LL, true>();              \
    return e != cudaSuccess ? e : prepare_fft_t<LL, false>(); \
  }
  switch (L) {
    ELF_PREP_CASE(16)
    ELF_PREP_CASE(32)
    ELF_PREP_CASE(64)
    ELF_PREP_CASE(128)
    ELF_PREP_CASE(256)
    ELF_PREP_CASE(512)
    ELF_PREP_CASE(1024)
    default:
      return cudaErrorInvalidValue;
  }
#undef ELF_PREP_CASE
}

cudaError_t launch_fft2(float2* data, int L, bool inverse, const float2* tw, cudaStream_t s) {
#define ELF_FFT_CASE(LL)                                                     \
  case LL:                                                                   \
    return inverse ? fft2_t<LL, true>(data, tw, s) : fft2_t<LL, false>(data, tw, s);
  switch (L) {
    ELF_FFT_CASE(16)
    ELF_FFT_CASE(32)
    ELF_FFT_CASE(64)
    ELF_FFT_CASE(128)
    ELF_FFT_CASE(256)
    ELF_FFT_CASE(512)
    ELF_FFT_CASE(1024)
    default:
      return cudaErrorInvalidValue;
  }
#undef ELF_FFT_CASE
}

__global__ void sign_scale_kernel(const float2* __restrict__ src, float2* __restrict__ dst, int L, float scale) {
  const size_t total = (size_t)L * L;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (size_t)y * L);
    const float sg = ((x + y) & 1) ? -scale : scale;
    const float2 v = src[i];
    dst[i] = make_float2(v.x * sg, v.y * sg);
  }
}

cudaError_t launch_sign_scale(const float2* src, float2* dst, int L, float scale, cudaStream_t s) {
  const size_t total = (size_t)L * L;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  sign_scale_kernel<<<blocks, 256, 0, s>>>(src, dst, L, scale);
  return cudaGetLastError();
}

}  // namespace elf
