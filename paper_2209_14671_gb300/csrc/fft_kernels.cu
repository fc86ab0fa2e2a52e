// Two-pass 2D FFT of an L x L complex array (the F_A of Eqs. 6-7, 13-14 and
// the object <-> spectrum maps).  Pass 1 transforms rows: each team of a CTA
// loads one row with coalesced float2 loads into shared memory, transforms it and
// writes it back.  Pass 2 transforms columns: a CTA loads an L x CW strip
// (coalesced CW-wide row segments), stores it column-major with a padded pitch,
// transforms each column and writes the strip back.
#include "fft.cuh"
#include "internal.cuh"

namespace elf {

// Rows (columns) per CTA: few for long transforms so that a 1024 x 1024 pass
// launches 512 (256) CTAs, more for short ones; one team of TL lanes each.
template <int L>
struct FftGrid {
  static constexpr int TL = FftTeam<L>::TL;
  static constexpr int RPC = (L >= 512) ? 2 : (L >= 256 ? 4 : 256 / TL);
  static constexpr int CPC = (L >= 512) ? 4 : (L >= 256 ? 8 : 256 / TL);
  static constexpr int ROW_THREADS = TL * RPC;
  static constexpr int COL_THREADS = TL * CPC;
  static constexpr size_t ROW_SMEM = 8 * ((size_t)L + (size_t)RPC * L);
  static constexpr size_t COL_SMEM = 8 * ((size_t)L + (size_t)CPC * (L + 1));
};

template <int L, bool INV>
__global__ void __launch_bounds__(FftGrid<L>::ROW_THREADS) fft_rows_kernel(float2* __restrict__ data,
                                                                             const float2* __restrict__ twg) {
  using G = FftGrid<L>;
  constexpr int NT = G::ROW_THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* rows = tw + L;
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += NT) tw[i] = twg[i];
  const int row0 = blockIdx.x * G::RPC;
  for (int i = tid; i < G::RPC * L; i += NT) {
    const int r = i / L, x = i - r * L;
    rows[r * L + x] = (row0 + r < L) ? data[(size_t)(row0 + r) * L + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int team = tid / G::TL, lane = tid % G::TL;
  team_fft<L, INV>(rows + team * L, tw, lane, row0 + team < L);
  __syncthreads();
  for (int i = tid; i < G::RPC * L; i += NT) {
    const int r = i / L, x = i - r * L;
    if (row0 + r < L) data[(size_t)(row0 + r) * L + x] = rows[r * L + x];
  }
}

template <int L, bool INV>
__global__ void __launch_bounds__(FftGrid<L>::COL_THREADS) fft_cols_kernel(float2* __restrict__ data,
                                                                             const float2* __restrict__ twg) {
  using G = FftGrid<L>;
  constexpr int NT = G::COL_THREADS;
  constexpr int CW = G::CPC;
  constexpr int LD = L + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* cols = tw + L;
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += NT) tw[i] = twg[i];
  const int c0 = blockIdx.x * CW;
  for (int i = tid; i < CW * L; i += NT) {
    const int y = i / CW, c = i - y * CW;
    cols[c * LD + y] = (c0 + c < L) ? data[(size_t)y * L + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int team = tid / G::TL, lane = tid % G::TL;
  team_fft<L, INV>(cols + team * LD, tw, lane, c0 + team < L);
  __syncthreads();
  for (int i = tid; i < CW * L; i += NT) {
    const int y = i / CW, c = i - y * CW;
    if (c0 + c < L) data[(size_t)y * L + c0 + c] = cols[c * LD + y];
  }
}

template <int L, bool INV>
static cudaError_t fft2_t(float2* data, const float2* tw, cudaStream_t s) {
  using G = FftGrid<L>;
  fft_rows_kernel<L, INV><<<(L + G::RPC - 1) / G::RPC, G::ROW_THREADS, G::ROW_SMEM, s>>>(data, tw);
  fft_cols_kernel<L, INV><<<(L + G::CPC - 1) / G::CPC, G::COL_THREADS, G::COL_SMEM, s>>>(data, tw);
  return cudaGetLastError();
}

template <int L, bool INV>
static cudaError_t prepare_fft_t() {
  using G = FftGrid<L>;
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::ROW_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_cols_kernel<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)G::COL_SMEM);
}

cudaError_t prepare_fft(int L) {
#define ELF_PREP_CASE(LL)                                     \
  case LL: {                                                  \
    cudaError_t e = prepare_fft_t<LL, true>();                \
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
