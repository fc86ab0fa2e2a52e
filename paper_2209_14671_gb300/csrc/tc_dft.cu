// Precision form: the per-LED tile transforms of Eqs. 1 and 9 as dense complex
// matrix products on the tensor cores (tcgen05, accumulators in tensor memory),
// for 128 x 128 tiles.  The paper has no counterpart; this is an alternative to
// the FP32 FFT of tile_kernel.cu, selected by elf_options.tile_dft.
//
// One iteration's tile path becomes, for all LEDs at once:
//   prep      X  = band block of P o M_n Psi                    (B x B, B = 64 >= band)
//   gemm 1    Y  = X E          rows: inverse DFT along x        (128 x 64) (64 x 128)
//   gemm 2    O~ = E^T Y        columns: inverse DFT along y     (128 x 64) (64 x 128)
//   stencil   W  from O~ and I_n (Eqs. 5, 12, 11), FP64 cost partials
//   gemm 3    Z  = F W          columns: forward DFT, band rows   (128 x 128) (128 x 128)
//   gemm 4    G~ = Z F^T        rows: forward DFT, band columns   (128 x 128) (128 x 64)
//   extract   G on the pupil support (compact order)
// E / F hold e^{+-2 pi i j x / n} for the band frequencies j only (the rest of the
// spectrum tile is zero or not needed), built in FP64 on the host.
//
// Each complex product C = A B is one real GEMM: [Ar Ai] [[Br Bi], [-Bi Br]], and
// each real operand x is split into BF16 x = hi + lo; C ~ Ah Bh + Ah Bl + Al Bh
// (three products concatenated along K), accumulated in FP32 in tensor memory.
// The MMA is tcgen05.mma.cta_group::1.kind::f16 with M = 128, N = 2 n_c, K = 16,
// operands in shared memory in the no-swizzle K-major layout (8-row x 16-byte core
// matrices; LBO = stride between core matrices along K, SBO = between 8-row
// groups), issued by one thread and completed through an mbarrier.  Every wait is
// bounded: on time-out the kernel sets an error flag, waits (bounded) for its own
// operations and frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace elf {

namespace {

constexpr int kTcThreads = 256;
constexpr int kChunk = 64;           // bf16 elements of K per pipeline stage
constexpr int kCoreLBO = 128;        // bytes between core matrices along K
constexpr int kCoreSBO = 1024;       // bytes between 8-row groups (8 core matrices of K per chunk)
constexpr long kSpinLimit = 1 << 22; // bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((kCoreLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kCoreSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: D fp32, A/B bf16, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(32);
  }
  return false;
}

// byte offset of element (row, k) of a K-major chunk (k < 64) in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * kCoreSBO + (k >> 3) * kCoreLBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

}  // namespace

// Batched complex GEMM C[b] = A[b] B[b] with M = 128, K = KC, N = NC (complex).
// Element (m, k) of A[b] at A + b*a.sAb + m*a.sAm + k*a.sAk (float2 units), rows
// m >= a.rowsA read as zero; likewise B (k, n) and C (m, n); rows m >= a.rowsC of C
// are not written.
struct CgemmArgs {
  const float2* A; long sAb, sAm, sAk; int rowsA;
  const float2* B; long sBb, sBk, sBn;
  float2* C; long sCb, sCm, sCn; int rowsC;
  int* err;
};

template <int KC, int NC>
__global__ void __launch_bounds__(kTcThreads) tc_cgemm_kernel(const CgemmArgs a) {
  constexpr int NR = 2 * NC;                 // real columns of D (<= 256)
  constexpr int KR = 6 * KC;                 // real K of the split product
  constexpr int NCH = KR / kChunk;           // pipeline chunks
  constexpr int A_BYTES = 128 * kChunk * 2;  // 16 KB
  constexpr int B_BYTES = NR * kChunk * 2;   // up to 32 KB
  static_assert(NR >= 32 && NR <= 256 && NR % 32 == 0, "N");
  static_assert((2 * KC) % kChunk == 0, "K");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA[2] = {smem, smem + A_BYTES + B_BYTES};
  unsigned char* sB[2] = {smem + A_BYTES, smem + 2 * A_BYTES + B_BYTES};
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * (A_BYTES + B_BYTES));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x;
  const float2* A = a.A + (long)b * a.sAb;
  const float2* B = a.B + (long)b * a.sBb;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(NR)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  for (int i = 0; i < NCH; ++i) {
    const int st = i & 1;
    if (i >= 2 && !mbar_wait(smem_u32(&mbar[st]), ((i - 2) >> 1) & 1)) ok = false;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    // chunk i covers real K indices [64 i, 64 i + 64): product term s, half h, complex k0
    const int q0 = i * kChunk;
    const int s = q0 / (2 * KC), h = (q0 % (2 * KC)) / KC, k0 = q0 % KC;
    const bool a_lo = (s == 2), b_lo = (s == 1);
    // operands are read along whichever of their indices is contiguous in memory
    const bool a_rows_fast = (a.sAm == 1), b_cols_fast = (a.sBn == 1);
    for (int e = tid; e < 128 * kChunk; e += kTcThreads) {
      int m, t;
      if (a_rows_fast) {
        t = e >> 7;
        m = e & 127;
      } else {
        m = e / kChunk;
        t = e - m * kChunk;
      }
      float v = 0.f;
      if (m < a.rowsA) {
        const float2 z = A[(long)m * a.sAm + (long)(k0 + t) * a.sAk];
        v = h ? z.y : z.x;
      }
      __nv_bfloat16 hi, lo;
      split_bf16(v, hi, lo);
      *reinterpret_cast<__nv_bfloat16*>(sA[st] + core_off(m, t)) = a_lo ? lo : hi;
    }
    for (int e = tid; e < NR * kChunk; e += kTcThreads) {
      int j, t;
      if (b_cols_fast) {
        t = e / NR;
        j = e - t * NR;
      } else {
        j = e / kChunk;
        t = e - j * kChunk;
      }
      const int n = (j < NC) ? j : j - NC;
      const float2 z = B[(long)(k0 + t) * a.sBk + (long)n * a.sBn];
      // [[Br Bi], [-Bi Br]]: first half of K pairs with Ar, second with Ai
      float v;
      if (j < NC) v = h ? -z.y : z.x;
      else v = h ? z.x : z.y;
      __nv_bfloat16 hi, lo;
      split_bf16(v, hi, lo);
      *reinterpret_cast<__nv_bfloat16*>(sB[st] + core_off(j, t)) = b_lo ? lo : hi;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t idesc = idesc_bf16(128, NR);
#pragma unroll
      for (int kk = 0; kk < kChunk / 16; ++kk) {
        const uint64_t ad = smem_desc(smem_u32(sA[st]) + kk * 2 * kCoreLBO);
        const uint64_t bd = smem_desc(smem_u32(sB[st]) + kk * 2 * kCoreLBO);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[st]))
                   : "memory");
    }
  }
  // the last commit covers every MMA issued before it
  if (ok && !mbar_wait(smem_u32(&mbar[(NCH - 1) & 1]), ((NCH - 1) >> 1) & 1)) ok = false;
  ok = __syncthreads_and(ok);
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // warps w and w + 4 share TMEM lane quadrant w % 4 and split the columns
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    float2* C = a.C + (long)b * a.sCb + (long)row * a.sCm;
    for (int cb = half * 32; cb < NC; cb += 64) {
      uint32_t re[32], im[32];
      const uint32_t tre = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)cb;
      const uint32_t tim = tre + (uint32_t)NC;
#define ELF_TMEM_LD(dst, addr)                                                                                    \
  asm volatile(                                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"            \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                              \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]), "=r"(dst[6]),       \
        "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]), "=r"(dst[12]), "=r"(dst[13]),    \
        "=r"(dst[14]), "=r"(dst[15]), "=r"(dst[16]), "=r"(dst[17]), "=r"(dst[18]), "=r"(dst[19]),                 \
        "=r"(dst[20]), "=r"(dst[21]), "=r"(dst[22]), "=r"(dst[23]), "=r"(dst[24]), "=r"(dst[25]),                 \
        "=r"(dst[26]), "=r"(dst[27]), "=r"(dst[28]), "=r"(dst[29]), "=r"(dst[30]), "=r"(dst[31])                  \
      : "r"(addr))
      ELF_TMEM_LD(re, tre);
      ELF_TMEM_LD(im, tim);
#undef ELF_TMEM_LD
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < a.rowsC) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          C[(long)(cb + j) * a.sCn] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
      }
    }
  } else if (tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NR) : "memory");
}

template <int KC, int NC>
static constexpr size_t cgemm_smem() {
  return 2 * (size_t)(128 * kChunk * 2 + 2 * NC * kChunk * 2) + 64;
}

template <int KC, int NC>
static cudaError_t cgemm(const CgemmArgs& a, int batch, cudaStream_t s) {
  tc_cgemm_kernel<KC, NC><<<batch, kTcThreads, cgemm_smem<KC, NC>(), s>>>(a);
  return cudaGetLastError();
}

template <int KC, int NC>
static cudaError_t cgemm_prepare() {
  return cudaFuncSetAttribute(tc_cgemm_kernel<KC, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cgemm_smem<KC, NC>());
}

// ---------------------------------------------------------------- helper kernels
// X[b][r][c] = P o M_b Psi on the band block (r, c < nb), zero elsewhere (64 x 64).
__global__ void tc_prep_kernel(const TcArgs a) {
  const int b = blockIdx.x;
  const int2 org = a.origin[b];
  for (int e = threadIdx.x; e < kTcBand * kTcBand; e += blockDim.x) {
    const int r = e / kTcBand, c = e - r * kTcBand;
    float2 v = make_float2(0.f, 0.f);
    if (r < a.nb && c < a.nb) {
      const int jy = a.Blo + r, jx = a.Blo + c;
      if ((unsigned)(jx - a.row_xs[jy]) < (unsigned)a.row_cnt[jy])
        v = cmul(a.pupil[jy * a.n + jx], a.psi[(size_t)(org.x + jy) * a.N + org.y + jx]);
    }
    a.X[(size_t)b * kTcBand * kTcBand + e] = v;
  }
}

// Residual, normaliser and W on the 128 x 128 spatial tile of LED b (Eqs. 5, 12, 11;
// Eq. 4/10 for the amplitude fidelity), with the (-1)^(x+y) shifts and the
// u^-2 n^-2 scale; FP64 cost partial per LED.
__global__ void __launch_bounds__(512) tc_stencil_kernel(const TcArgs a) {
  constexpr int n = kTcN;
  extern __shared__ float s_f[];
  float* R = s_f;                 // n x n residual
  float* WX = R + n * n;          // n x n omega_x
  float* WY = WX + n * n;         // n x n omega_y
  __shared__ float red[2 * 16];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float2* O = a.O + (size_t)b * n * n;
  const float* I = a.meas + (size_t)b * n * n;
  for (int p = tid; p < n * n; p += blockDim.x) {
    const int y = p / n, x = p - y * n;
    float2 o = O[p];
    const float sg = ((x + y) & 1) ? -a.scale : a.scale;
    o = make_float2(o.x * sg, o.y * sg);
    const float m2 = cabs2(o);
    R[p] = (a.fidelity == 0) ? (m2 - I[p]) : (sqrtf(m2) - sqrtf(fmaxf(I[p], 0.f)));
  }
  __syncthreads();
  const float tau = a.tau, tau2 = fmaxf(a.tau * a.tau, 1e-36f), hit = (a.tau > 0.f) ? 0.5f / a.tau : 0.f;
  float acc = 0.f;
  for (int p = tid; p < n * n; p += blockDim.x) {
    const int y = p / n, x = p - y * n;
    const float dx = (x < n - 1) ? R[p + 1] - R[p] : 0.f;
    const float dy = (y < n - 1) ? R[p + n] - R[p] : 0.f;
    float wx, wy, phi;
    if (a.iso) {
      const float ss = dx * dx + dy * dy;
      const float inv = rsqrtf(fmaxf(ss, tau2));
      wx = dx * inv;
      wy = dy * inv;
      phi = (ss >= tau * tau) ? ss * inv : ss * hit + 0.5f * tau;
    } else {
      const float ax = fabsf(dx), ay = fabsf(dy);
      wx = dx / fmaxf(ax, tau);
      wy = dy / fmaxf(ay, tau);
      phi = ((ax >= tau) ? ax : ax * ax * hit + 0.5f * tau) + ((ay >= tau) ? ay : ay * ay * hit + 0.5f * tau);
    }
    WX[p] = wx;
    WY[p] = wy;
    acc += phi;
  }
  __syncthreads();
  for (int p = tid; p < n * n; p += blockDim.x) {
    const int y = p / n, x = p - y * n;
    float w = -WX[p] - WY[p];
    if (x >= 1) w += WX[p - 1];
    if (y >= 1) w += WY[p - n];
    float2 o = O[p];
    const float sg = ((x + y) & 1) ? -a.scale : a.scale;
    o = make_float2(o.x * sg, o.y * sg);
    float f = w;
    if (a.fidelity != 0) f = w / (2.f * fmaxf(sqrtf(cabs2(o)), a.eta));
    if ((x + y) & 1) f = -f;
    a.Wt[(size_t)b * n * n + p] = cscale(o, f);
  }
  const float part[1] = {acc};
  double sum[1];
  block_sum_ff<1>(part, red, sum);
  if (tid == 0) a.costpart[b] = sum[0];
}

// G on the support (compact order) from the band block G~ (64 x 64), times u^-2 n^-2.
__global__ void tc_extract_kernel(const TcArgs a) {
  const int b = blockIdx.x;
  for (int e = threadIdx.x; e < a.nb * a.nb; e += blockDim.x) {
    const int r = e / a.nb, c = e - r * a.nb;
    const int jy = a.Blo + r, jx = a.Blo + c;
    const int d = jx - a.row_xs[jy];
    if ((unsigned)d < (unsigned)a.row_cnt[jy])
      a.G[(size_t)b * a.S + a.row_off[jy] + d] = cscale(a.Gt[(size_t)b * kTcBand * kTcBand + r * kTcBand + c], a.scale);
  }
}

cudaError_t prepare_tc() {
  cudaError_t e = cgemm_prepare<kTcBand, kTcN>();
  if (e == cudaSuccess) e = cgemm_prepare<kTcN, kTcN>();
  if (e == cudaSuccess) e = cgemm_prepare<kTcN, kTcBand>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             3 * kTcN * kTcN * (int)sizeof(float));
  return e;
}

cudaError_t launch_tc_tile(const TcArgs& a, cudaStream_t s) {
  const int K = a.K;
  const long B2 = (long)kTcBand * kTcBand, NN = (long)kTcN * kTcN;
  tc_prep_kernel<<<K, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CgemmArgs g{};
  g.err = a.err;
  // gemm 1: Y (64 x 128) = X (64 x 64) E (64 x 128); M padded to 128 with zero rows
  g.A = a.X; g.sAb = B2; g.sAm = kTcBand; g.sAk = 1; g.rowsA = kTcBand;
  g.B = a.Einv; g.sBb = 0; g.sBk = kTcN; g.sBn = 1;
  g.C = a.Y; g.sCb = (long)kTcBand * kTcN; g.sCm = kTcN; g.sCn = 1; g.rowsC = kTcBand;
  if ((e = cgemm<kTcBand, kTcN>(g, K, s)) != cudaSuccess) return e;
  // gemm 2: O~ (128 x 128) = E^T (128 x 64) Y (64 x 128)
  g.A = a.Einv; g.sAb = 0; g.sAm = 1; g.sAk = kTcN; g.rowsA = kTcN;
  g.B = a.Y; g.sBb = (long)kTcBand * kTcN; g.sBk = kTcN; g.sBn = 1;
  g.C = a.O; g.sCb = NN; g.sCm = kTcN; g.sCn = 1; g.rowsC = kTcN;
  if ((e = cgemm<kTcBand, kTcN>(g, K, s)) != cudaSuccess) return e;
  tc_stencil_kernel<<<K, 512, 3 * kTcN * kTcN * sizeof(float), s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // gemm 3: Z (64 x 128) = F (64 x 128) W (128 x 128)
  g.A = a.Ffwd; g.sAb = 0; g.sAm = kTcN; g.sAk = 1; g.rowsA = kTcBand;
  g.B = a.Wt; g.sBb = NN; g.sBk = kTcN; g.sBn = 1;
  g.C = a.Z; g.sCb = (long)kTcBand * kTcN; g.sCm = kTcN; g.sCn = 1; g.rowsC = kTcBand;
  if ((e = cgemm<kTcN, kTcN>(g, K, s)) != cudaSuccess) return e;
  // gemm 4: G~ (64 x 64) = Z (64 x 128) F^T (128 x 64)
  g.A = a.Z; g.sAb = (long)kTcBand * kTcN; g.sAm = kTcN; g.sAk = 1; g.rowsA = kTcBand;
  g.B = a.Ffwd; g.sBb = 0; g.sBk = 1; g.sBn = kTcN;
  g.C = a.Gt; g.sCb = B2; g.sCm = kTcBand; g.sCn = 1; g.rowsC = kTcBand;
  if ((e = cgemm<kTcN, kTcBand>(g, K, s)) != cudaSuccess) return e;
  tc_extract_kernel<<<K, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace elf
