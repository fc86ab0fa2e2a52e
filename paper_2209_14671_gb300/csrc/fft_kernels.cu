// 2D FFT of an L x L complex array (the F_A of Eqs. 6-7, 13-14 and the object <-> spectrum maps).
// Rows: each team of a CTA loads one row with coalesced float2 loads, transforms it and writes it
// back.  Columns, with a scratch array (the L x L transforms of the iteration): the four-step split
// L = P * Q of the column index in two passes without shared memory, one thread per (column,
// sub-transform) and a warp on 32 adjacent columns, so every access is a whole row segment:
//   pass A  thread (x, n2): the P-point DFT over rows Q n1 + n2 (n1 < P), times W_L^(n2 k1),
//           into scratch rows n2 P + k1;
//   pass B  thread (x, k1): the Q-point DFT over scratch rows n2 P + k1 (n2 < Q), giving
//           X[k1 + P k2] in row k1 + P k2.
// Without a scratch array a CTA loads an L x CW strip (coalesced CW-wide row segments), stores it
// column-major with a padded pitch, transforms each column and writes the strip back.
#include "fft.cuh"
#include "internal.cuh"

namespace elf {

// Rows per CTA: few for long transforms so that a 1024 x 1024 pass launches 256 CTAs, more for
// short ones; one team of TL lanes each.  Column CTAs have as many teams but twice the columns
// (each team transforms two), so the row segments they load and store are twice as long (64 bytes
// for 1024 x 1024) while their registers still fit beside a tile-kernel CTA.
template <int L>
struct FftGrid {
  static constexpr int TL = FftTeam<L>::TL;
  static constexpr int PL = FftTeam<L>::PADDED;
  static constexpr int RPC = (128 / TL < L) ? 128 / TL : L;  // rows per CTA (one team each)
  static constexpr int CTEAMS = (128 / TL < L) ? 128 / TL : L;  // teams of a column CTA
  static constexpr int CPC = (2 * CTEAMS <= L) ? 2 * CTEAMS : CTEAMS;  // columns per CTA
  static constexpr int ROW_THREADS = TL * RPC;
  static constexpr int COL_THREADS = TL * CTEAMS;
  static constexpr int LD = PL + 1;               // column pitch (odd)
  static constexpr size_t ROW_SMEM = 8 * ((size_t)L + (size_t)RPC * PL);
  static_assert(L % CPC == 0 && L % RPC == 0, "rows and columns per CTA divide L");
  static constexpr size_t COL_SMEM = 8 * ((size_t)L + (size_t)CPC * LD);
};

// Rows pass: each team transforms one row, reading its pass-1 inputs straight
// from global memory into registers (coalesced across lanes, all loads in
// flight at once) and writing its pass-2 outputs straight back; shared memory
// only carries the transpose between the two passes.  src may be data (in place) or another
// array of the same shape (out of place): a row is read whole before it is written.
template <int L, bool INV>
__global__ void __launch_bounds__(FftGrid<L>::ROW_THREADS) fft_rows_kernel(const float2* src, float2* data,
                                                                             const float2* __restrict__ twg) {
  using G = FftGrid<L>;
  using T = FftTeam<L>;
  constexpr int NT = G::ROW_THREADS;
  constexpr int P = T::P, Q = T::Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* rows = tw + L;
  const int tid = threadIdx.x;
  const int team = tid / Q, lane = tid % Q;
  const int row = blockIdx.x * G::RPC + team;
  const bool act = row < L;
  float2* g = data + (size_t)(act ? row : 0) * L;
  const float2* gs = src + (size_t)(act ? row : 0) * L;
  pdl_launch_dependents();
  pdl_wait();  // the previous kernel of a chain wrote src
  float2 v[P];
  if (act) {
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = gs[lane + Q * j];
  }
  for (int i = tid; i < L; i += NT) tw[i] = twg[i];
  __syncthreads();
  float2* buf = rows + team * G::PL;
  if (act) {
    Dft<P, INV>::run(v);
#pragma unroll
    for (int k = 1; k < P; ++k) {
      float2 w = tw[k * Q + lane];
      if (INV) w.y = -w.y;
      v[k] = cmul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) buf[k * (Q + 1) + lane] = v[k];
  }
  __syncwarp();
  if (act) {
#pragma unroll
    for (int m = 0; m < P / Q; ++m) {
      const int k1 = lane + Q * m;
#pragma unroll
      for (int l = 0; l < Q; ++l) v[m * Q + l] = buf[k1 * (Q + 1) + l];
      Dft<Q, INV>::run(v + m * Q);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) g[k1 + P * k2] = v[m * Q + k2];
    }
  }
}

template <int L, bool INV>
__global__ void __launch_bounds__(FftGrid<L>::COL_THREADS) fft_cols_kernel(float2* __restrict__ data,
                                                                             const float2* __restrict__ twg) {
  using G = FftGrid<L>;
  constexpr int NT = G::COL_THREADS;
  constexpr int CW = G::CPC;
  constexpr int LD = G::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* cols = tw + L;
  const int tid = threadIdx.x;
  pdl_launch_dependents();
  for (int i = tid; i < L; i += NT) tw[i] = twg[i];
  const int c0 = blockIdx.x * CW;
  pdl_wait();  // the rows pass wrote data
  // asynchronous 8-byte copies, all in flight at once (CW divides L, so c0 + c < L)
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(cols);
  for (int i = tid; i < CW * L; i += NT) {
    const int y = i / CW, c = i - y * CW;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sbase + 8u * (c * LD + FftTeam<L>::pidx(y))),
                 "l"(data + (size_t)y * L + c0 + c)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int team = tid / G::TL, lane = tid % G::TL;
#pragma unroll 1  // one column's values in registers at a time
  for (int c = team; c < CW; c += G::CTEAMS) team_fft<L, INV>(cols + c * LD, tw, lane, true);  // same count per team
  __syncthreads();
  for (int i = tid; i < CW * L; i += NT) {
    const int y = i / CW, c = i - y * CW;
    data[(size_t)y * L + c0 + c] = cols[c * LD + FftTeam<L>::pidx(y)];
  }
}

// Column passes of the four-step split (see the top of the file); blocks of 32 columns x 4 sub-transforms.
// twg[k1 * Q + n2] = W_L^(n2 k1) (forward sign), the team twiddle table of fft.cuh.
template <int L, bool INV>
__global__ void __launch_bounds__(128) fft_cols_a_kernel(const float2* __restrict__ data, float2* __restrict__ tmp,
                                                         const float2* __restrict__ twg) {
  constexpr int P = FftTeam<L>::P, Q = FftTeam<L>::Q;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int n2 = blockIdx.y * 4 + threadIdx.y;
  pdl_launch_dependents();
  pdl_wait();  // the rows pass wrote data
  float2 v[P];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) v[n1] = data[(size_t)(Q * n1 + n2) * L + x];
  Dft<P, INV>::run(v);
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    float2 w = twg[k1 * Q + n2];
    if (INV) w.y = -w.y;
    tmp[(size_t)(n2 * P + k1) * L + x] = k1 ? cmul(v[k1], w) : v[k1];
  }
}

template <int L, bool INV>
__global__ void __launch_bounds__(128) fft_cols_b_kernel(const float2* __restrict__ tmp, float2* __restrict__ data) {
  constexpr int P = FftTeam<L>::P, Q = FftTeam<L>::Q;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int k1 = blockIdx.y * 4 + threadIdx.y;
  pdl_launch_dependents();
  pdl_wait();  // pass A wrote tmp (and read data, which this pass overwrites)
  float2 v[Q];
#pragma unroll
  for (int n2 = 0; n2 < Q; ++n2) v[n2] = tmp[(size_t)(n2 * P + k1) * L + x];
  Dft<Q, INV>::run(v);
#pragma unroll
  for (int k2 = 0; k2 < Q; ++k2) data[(size_t)(k1 + P * k2) * L + x] = v[k2];
}

// With pdl, the column pass (and the rows pass when `dep`: it follows another kernel of the stream)
// starts early by programmatic dependent launch and waits for its predecessor inside.
template <typename... P, typename... A>
static cudaError_t launch_maybe_dependent(bool pdl, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                          A... args) {
  if (pdl) return launch_dependent(k, grid, block, smem, s, args...);
  k<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}

template <int L, bool INV>
static cudaError_t fft2_t(float2* data, const float2* tw, cudaStream_t s, const float2* src, float2* tmp, bool dep,
                          bool pdl) {
  using G = FftGrid<L>;
  const float2* in = src ? src : data;
  cudaError_t e;
  if (dep && pdl) {
    e = launch_dependent(fft_rows_kernel<L, INV>, dim3((L + G::RPC - 1) / G::RPC), dim3(G::ROW_THREADS), G::ROW_SMEM, s,
                         in, data, tw);
  } else {
    fft_rows_kernel<L, INV><<<(L + G::RPC - 1) / G::RPC, G::ROW_THREADS, G::ROW_SMEM, s>>>(in, data, tw);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  if constexpr (L >= 512) {  // at 256 the strip kernel's one launch is faster (64/256/49: 28.5 vs 29.1 us)
    if (tmp) {
      constexpr int P = FftTeam<L>::P, Q = FftTeam<L>::Q;
      const float2* d = data;
      const float2* t = tmp;
      e = launch_maybe_dependent(pdl, fft_cols_a_kernel<L, INV>, dim3(L / 32, Q / 4), dim3(32, 4), 0, s, d, tmp, tw);
      if (e == cudaSuccess)
        e = launch_maybe_dependent(pdl, fft_cols_b_kernel<L, INV>, dim3(L / 32, P / 4), dim3(32, 4), 0, s, t, data);
      return e;
    }
  }
  return launch_maybe_dependent(pdl, fft_cols_kernel<L, INV>, dim3((L + G::CPC - 1) / G::CPC), dim3(G::COL_THREADS),
                                G::COL_SMEM, s, data, tw);
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

cudaError_t launch_fft2(float2* data, int L, bool inverse, const float2* tw, cudaStream_t s, const float2* src,
                        float2* tmp, bool dep, bool pdl) {
#define ELF_FFT_CASE(LL)                                                        \
  case LL:                                                                      \
    return inverse ? fft2_t<LL, true>(data, tw, s, src, tmp, dep, pdl)          \
                   : fft2_t<LL, false>(data, tw, s, src, tmp, dep, pdl);
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
