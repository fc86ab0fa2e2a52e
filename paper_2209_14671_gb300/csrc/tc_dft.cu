// Precision form: the per-LED tile transforms of Eqs. 1 and 9 as dense complex
// matrix products on the tensor cores (tcgen05, accumulators in tensor memory),
// for 128 x 128 tiles.  The paper has no counterpart; this is an alternative to
// the FP32 FFT of tile_kernel.cu, selected by elf_options.tile_dft.
//
// One iteration's tile path, for all LEDs at once (j: band index, x, y: pixel,
// k: band frequency of the forward transform; every product's contraction index
// is the column index of the operand the previous step stored, so no step
// transposes anything):
//   prep    X[j_y][j_x]   = band block of P o M_n Psi (64 x 64)
//   gemm 1  Y'[x][j_y]    = sum_jx E[j_x][x] X[j_y][j_x]      (Y transposed, 128 x 64)
//   gemm 2  O'[x][y]      = sum_jy Y'[x][j_y] E[j_y][y]       (o transposed, 128 x 128)
//   stencil W'[x][y] from O' and I_n (Eqs. 5, 12, 11), FP64-accurate cost partials
//   gemm 3  Z[k_y][x]     = sum_y F[k_y][y] W'[x][y]          (64 x 128)
//   gemm 4  G[k_y][k_x]   = sum_x Z[k_y][x] F[k_x][x]         (64 x 64), support pixels to G
// E / F hold e^{+-2 pi i (Blo + j) x / n} for the band frequencies only (built in
// FP64 on the host).
//
// Arithmetic: each complex product is a real GEMM with the data operand stacked
// along K as [re | im] and the constant operand expanded, either as two A
// matrices [Cr, -Ci] and [Ci, Cr] (real and imaginary outputs in two tensor-memory
// column ranges) or as one B matrix [[Cr, Ci], [-Ci, Cr]] (real and imaginary
// columns side by side).  Every real operand is split into BF16 hi + lo and the
// product taken as hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory.
//
// Operands live in global memory as "images": for each 64-wide chunk of K, the
// hi plane then the lo plane, each R rows x 64 BF16 in the no-swizzle K-major
// core-matrix layout the MMA reads from shared memory (8-row x 16-byte core
// matrices; 128 bytes between core matrices along K, 1024 bytes between 8-row
// groups).  A chunk plane is one contiguous block of R x 128 bytes, moved into
// shared memory by one bulk copy.  The constants' images are built on the host;
// each kernel that produces a data operand writes it as an image.
//
// GEMM kernel: one CTA of 256 threads per LED, M = 128, a two-stage pipeline of
// K chunks: warp 0 issues the bulk copies (completion counted in bytes on a "full"
// mbarrier), warp 1 issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate) and
// commits each stage to an "empty" mbarrier; all warps read the accumulators
// (tcgen05.ld) for the epilogue.  Every wait is bounded: on time-out the kernel
// sets the error flag, stops issuing, waits (bounded) for what it issued and frees
// its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace elf {

namespace {

constexpr int kTcThreads = 256;
constexpr int kCoreLBO = 128;         // bytes between core matrices along K
constexpr int kCoreSBO = 1024;        // bytes between 8-row groups
constexpr long kSpinLimit = 1L << 18; // bounded waits: about 1 s of mbarrier polls (3.8 us per poll, measured)

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

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// one contiguous global -> shared copy, counted on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// byte offset of element (row, k) of one chunk plane (k < 64) in the core-matrix layout
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * kCoreSBO + (k >> 3) * kCoreLBO + (row & 7) * 16 + (k & 7) * 2);
}

// BF16 hi/lo split of a float: v = hi + lo to about 16 significant bits
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Writes eight consecutive K values (k0 multiple of 8) of row `row` into an image of R rows:
// one 16-byte store per plane.
__device__ __forceinline__ void put8(unsigned char* img, int R, int row, int k0, const float (&v)[8]) {
  __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split_bf16(v[i], hi[i], lo[i]);
  const size_t plane = (size_t)R * 128;
  unsigned char* base = img + (size_t)(k0 >> 6) * 2 * plane + core_off(row, k0 & 63);
  *reinterpret_cast<uint4*>(base) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(base + plane) = *reinterpret_cast<const uint4*>(lo);
}

}  // namespace

// ------------------------------------------------------------------ batched GEMM on images
// D = sum over K of A (128 rows) times B (RB rows), per LED b = blockIdx.x:
//   A = g.A + b * g.sA (and, with NA = 2, a second A image g.A2off bytes further on: real and
//   imaginary outputs in tensor-memory columns [0, RB) and [RB, 2 RB)); B = g.B + b * g.sB.
// Epilogue MODE: kImage writes row r of the accumulator (all NA * RB columns, in order, as K)
// into the image g.out (128 rows) of LED b; kOT writes O'[x = r][y] = (D[y], D[128 + y]) as
// float2; kG writes the support pixels of G from G[k_y = r][k_x] = (D[k_x], D[64 + k_x]).
enum { kImage = 0, kOT = 1, kG = 2 };

struct TcGemmArgs {
  const unsigned char* A;
  long sA, A2off;
  const unsigned char* B;
  long sB;
  unsigned char* out;  // kImage: output images
  long sOut;
  TcArgs t;            // kOT / kG outputs and the support tables
};

template <int NA, int RB, int KR>
struct GemmShape {
  static constexpr int NCH = KR / 64;                  // K chunks
  static constexpr int S = 2;                          // pipeline stages
  static constexpr uint32_t PA = 128 * 128;            // bytes of one A chunk plane
  static constexpr uint32_t PB = RB * 128;             // bytes of one B chunk plane
  static constexpr uint32_t STAGE = NA * 2 * PA + 2 * PB;
  static constexpr int NCOL = NA * RB;                 // tensor-memory columns
  static constexpr size_t SMEM = S * (size_t)STAGE + 64;
  static_assert(NCOL == 32 || NCOL == 64 || NCOL == 128 || NCOL == 256, "tensor-memory allocation");
  static_assert(RB % 16 == 0 && RB >= 16 && RB <= 256, "N of kind::f16 with M = 128");
  static_assert(KR % 64 == 0, "K chunks");
};

#define ELF_TMEM_LD32(dst, addr)                                                                                  \
  asm volatile(                                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"            \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                              \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]), "=r"(dst[6]),       \
        "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]), "=r"(dst[12]), "=r"(dst[13]),    \
        "=r"(dst[14]), "=r"(dst[15]), "=r"(dst[16]), "=r"(dst[17]), "=r"(dst[18]), "=r"(dst[19]),                 \
        "=r"(dst[20]), "=r"(dst[21]), "=r"(dst[22]), "=r"(dst[23]), "=r"(dst[24]), "=r"(dst[25]),                 \
        "=r"(dst[26]), "=r"(dst[27]), "=r"(dst[28]), "=r"(dst[29]), "=r"(dst[30]), "=r"(dst[31])                  \
      : "r"(addr))

template <int NA, int RB, int KR, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcGemmArgs g) {
  using Sh = GemmShape<NA, RB, KR>;
  constexpr int NCH = Sh::NCH, S = Sh::S, NCOL = Sh::NCOL;
  constexpr uint32_t PA = Sh::PA, PB = Sh::PB, STAGE = Sh::STAGE;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x;
  const unsigned char* A = g.A + (size_t)b * g.sA;
  const unsigned char* B = g.B + (size_t)b * g.sB;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: chunk c into stage c % S once the MMAs of chunk c - S have released it
    int c = 0;
    for (; c < NCH; ++c) {
      const int s = c % S;
      if (c >= S && !mbar_wait(&empty[s], ((c / S) - 1) & 1)) {
        atomicExch(g.t.err, 1);
        break;
      }
      mbar_expect_tx(&full[s], STAGE);
      unsigned char* st = smem + (size_t)s * STAGE;
#pragma unroll
      for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int p = 0; p < 2; ++p)
          bulk_copy(st + (a * 2 + p) * PA, A + a * g.A2off + (size_t)(c * 2 + p) * PA, PA, &full[s]);
#pragma unroll
      for (int p = 0; p < 2; ++p) bulk_copy(st + NA * 2 * PA + p * PB, B + (size_t)(c * 2 + p) * PB, PB, &full[s]);
    }
    // every copy issued has landed before the CTA may end (immediate when the MMAs consumed them)
    for (int i = (c > S ? c - S : 0); i < c; ++i)
      if (!mbar_wait(&full[i % S], (i / S) & 1)) atomicExch(g.t.err, 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K-steps of 16 per chunk, three BF16 products each (hi hi, hi lo, lo hi)
    const uint32_t idesc = idesc_bf16(128, RB);
    for (int c = 0; c < NCH; ++c) {
      const int s = c % S;
      if (!mbar_wait(&full[s], (c / S) & 1)) {
        atomicExch(g.t.err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t st = smem_u32(smem + (size_t)s * STAGE);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int pa = (t == 2) ? 1 : 0, pb = (t == 1) ? 1 : 0;
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const uint64_t ad = smem_desc(st + (a * 2 + pa) * PA + kk * 2 * kCoreLBO);
            const uint64_t bd = smem_desc(st + NA * 2 * PA + pb * PB + kk * 2 * kCoreLBO);
            const uint32_t acc = (c > 0 || kk > 0 || t > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(a * RB)),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    // completes when every MMA issued above has
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(done))
                 : "memory");
  }
  __syncwarp();
  bool ok = mbar_wait(done, 0);
  ok = __syncthreads_and(ok);
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // warps w and w + 4 share tensor-memory lane quadrant w % 4 (rows 32 q .. 32 q + 31)
    const int quad = warp & 3, half = warp >> 2;
    const int r = quad * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
    if constexpr (MODE == kImage) {
      unsigned char* img = g.out + (size_t)b * g.sOut;
      for (int c0 = half * 32; c0 < NCOL; c0 += 64) {
        uint32_t v[32];
        ELF_TMEM_LD32(v, trow + (uint32_t)c0);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          float f[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) f[i] = __uint_as_float(v[8 * o + i]);
          put8(img, 128, r, c0 + 8 * o, f);
        }
      }
    } else if constexpr (MODE == kOT) {
      float2* Ot = g.t.Ot + (size_t)b * kTcN * kTcN + (size_t)r * kTcN;
      for (int y0 = half * 32; y0 < kTcN; y0 += 64) {
        uint32_t re[32], im[32];
        ELF_TMEM_LD32(re, trow + (uint32_t)y0);
        ELF_TMEM_LD32(im, trow + (uint32_t)(kTcN + y0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; i += 2)
          *reinterpret_cast<float4*>(Ot + y0 + i) =
              make_float4(__uint_as_float(re[i]), __uint_as_float(im[i]), __uint_as_float(re[i + 1]),
                          __uint_as_float(im[i + 1]));
      }
    } else {  // kG: G on the support of band row r
      const int kx0 = half * 32;
      uint32_t re[32], im[32];
      ELF_TMEM_LD32(re, trow + (uint32_t)kx0);
      ELF_TMEM_LD32(im, trow + (uint32_t)(kTcBand + kx0));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (r < g.t.nb) {
        const int ky = g.t.Blo + r;
        const int xs = g.t.row_xs[ky], cnt = g.t.row_cnt[ky];
        float2* dst = g.t.G + (size_t)b * g.t.S + g.t.row_off[ky];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int d = g.t.Blo + kx0 + i - xs;
          if ((unsigned)d < (unsigned)cnt)
            dst[d] = make_float2(__uint_as_float(re[i]) * g.t.scale, __uint_as_float(im[i]) * g.t.scale);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(g.t.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
}

// ------------------------------------------------------------------ producers of data images
// X image (64 rows j_y, K = [Re X | Im X] over j_x): the band block of P o M_b Psi, zero outside
// the support.
__global__ void __launch_bounds__(256) tc_prep_kernel(const TcArgs a) {
  const int b = blockIdx.x;
  const int2 org = a.origin[b];
  unsigned char* img = a.iX + (size_t)b * kTcImgX;
  for (int e = threadIdx.x; e < kTcBand * (kTcBand / 8); e += blockDim.x) {
    const int r = e >> 3, c0 = (e & 7) * 8;
    float re[8], im[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + i;
      float2 v = make_float2(0.f, 0.f);
      if (r < a.nb && c < a.nb) {
        const int jy = a.Blo + r, jx = a.Blo + c;
        if ((unsigned)(jx - a.row_xs[jy]) < (unsigned)a.row_cnt[jy])
          v = cmul(a.pupil[jy * a.n + jx], a.psi[(size_t)(org.x + jy) * a.N + org.y + jx]);
      }
      re[i] = v.x;
      im[i] = v.y;
    }
    put8(img, kTcBand, r, c0, re);
    put8(img, kTcBand, r, kTcBand + c0, im);
  }
}

// Residual, normaliser and W on the 128 x 128 spatial tile of LED b (Eqs. 5, 12, 11; Eq. 4/10
// for the amplitude fidelity; the Sec. 6.3 power and log maps for fidelity 2 and 3) from o' = O'[x][y] (the transposed raw IDFT) times u^-2 n^-2.
// W' = o' f needs no (-1)^(x+y) factor: the inverse shift's sign and the forward shift's sign
// multiply to 1.  W' goes to the image of gemm 3's B (128 rows x, K = [Re W' | Im W'] over y);
// FP64-accurate cost partial per LED.
__global__ void __launch_bounds__(1024) tc_stencil_kernel(const TcArgs a) {
  constexpr int n = kTcN, P = n + 1;  // shared-memory pitch: columns and rows both conflict-free
  extern __shared__ float s_f[];
  float* R = s_f;          // residual, R[y * P + x]
  float* WX = R + n * P;   // omega_x
  float* WY = WX + n * P;  // omega_y
  __shared__ float red[2 * 32];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float2* Ot = a.Ot + (size_t)b * n * n;
  const float* I = a.meas + (size_t)b * n * n;
  const float scale = a.scale;
  for (int p = tid; p < n * n; p += blockDim.x) R[(p / n) * P + (p % n)] = I[p];
  __syncthreads();
  for (int p = tid; p < n * n; p += blockDim.x) {  // p = x n + y: O' read along y
    const int x = p / n, y = p - x * n;
    const float2 o = Ot[p];
    const float m2 = (o.x * o.x + o.y * o.y) * (scale * scale);
    const float meas = R[y * P + x];
    float r;
    if (a.fidelity == 0) {
      r = m2 - meas;
    } else if (a.fidelity == 1) {
      r = sqrtf(m2) - meas;  // meas holds sqrt(max(I, 0))
    } else {  // Sec. 6.3 maps: meas already holds g(max(I, 0))
      r = ((a.fidelity == 2) ? powf(m2, a.gexp) : log1pf(m2)) - meas;
    }
    R[y * P + x] = r;
  }
  __syncthreads();
  const float tau = a.tau, tau2 = fmaxf(a.tau * a.tau, 1e-36f), hit = (a.tau > 0.f) ? 0.5f / a.tau : 0.f;
  float acc = 0.f;
  for (int p = tid; p < n * n; p += blockDim.x) {
    const int y = p / n, x = p - y * n;
    const float r0 = R[y * P + x];
    const float dx = (x < n - 1) ? R[y * P + x + 1] - r0 : 0.f;
    const float dy = (y < n - 1) ? R[(y + 1) * P + x] - r0 : 0.f;
    float wx, wy, phi;
    if (a.iso) {
      const float ss = dx * dx + dy * dy;
      const float inv = rsqrtf(fmaxf(ss, tau2));
      wx = dx * inv;
      wy = dy * inv;
      phi = (ss >= tau * tau) ? ss * inv : ss * hit + 0.5f * tau;
    } else {
      const float ax = fabsf(dx), ay = fabsf(dy);
      wx = dx / fmaxf(ax, fmaxf(tau, 1e-18f));  // 0 at the origin when tau = 0
      wy = dy / fmaxf(ay, fmaxf(tau, 1e-18f));
      phi = ((ax >= tau) ? ax : ax * ax * hit + 0.5f * tau) + ((ay >= tau) ? ay : ay * ay * hit + 0.5f * tau);
    }
    WX[y * P + x] = wx;
    WY[y * P + x] = wy;
    acc += phi;
  }
  __syncthreads();
  unsigned char* img = a.iW + (size_t)b * kTcImgW;
  for (int e = tid; e < n * (n / 8); e += blockDim.x) {  // x fastest: conflict-free column reads
    const int x = e % n, y0 = (e / n) * 8;
    float re[8], im[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int y = y0 + i;
      float w = -WX[y * P + x] - WY[y * P + x];
      if (x >= 1) w += WX[y * P + x - 1];
      if (y >= 1) w += WY[(y - 1) * P + x];
      const float2 o = Ot[(size_t)x * n + y];
      const float2 os = make_float2(o.x * scale, o.y * scale);
      float f = w;
      if (a.fidelity == 1) f = w / (2.f * fmaxf(sqrtf(cabs2(os)), a.eta));
      if (a.fidelity == 2) f = w * a.gexp * powf(fmaxf(cabs2(os), a.eta * a.eta), a.gexp - 1.f);
      if (a.fidelity == 3) f = w / (cabs2(os) + 1.f);
      re[i] = os.x * f;
      im[i] = os.y * f;
    }
    put8(img, n, x, y0, re);
    put8(img, n, x, n + y0, im);
  }
  const float part[1] = {acc};
  double sum[1];
  block_sum_ff<1>(part, red, sum);
  if (tid == 0) a.costpart[b] = sum[0];
}

// ------------------------------------------------------------------ host: constant images
namespace {

uint16_t bf16_bits(float f) {  // round to nearest even (the operands are finite)
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// image of an R x KR real matrix val(row, k), split hi + lo from FP64
template <typename F>
void put_image(unsigned char* img, int R, int KR, F val) {
  const size_t plane = (size_t)R * 128;
  for (int row = 0; row < R; ++row)
    for (int k = 0; k < KR; ++k) {
      const double v = val(row, k);
      const uint16_t hi = bf16_bits((float)v);
      const uint16_t lo = bf16_bits((float)(v - (double)bf16_value(hi)));
      unsigned char* base = img + (size_t)(k >> 6) * 2 * plane + core_off(row, k & 63);
      std::memcpy(base, &hi, 2);
      std::memcpy(base + plane, &lo, 2);
    }
}

}  // namespace

std::vector<unsigned char> tc_constant_image(int which, int Blo, int nb) {
  constexpr int n = kTcN, nbp = kTcBand;
  const double pi = 3.14159265358979323846;
  // band DFT factors: e^{+i t} (inverse, E) and e^{-i t} (forward, F), t = 2 pi (Blo + j) x / n
  auto ang = [&](int j, int x) { return 2.0 * pi * (double)(((long)(Blo + j) * x) % n) / (double)n; };
  auto Er = [&](int j, int x) { return j < nb ? std::cos(ang(j, x)) : 0.0; };
  auto Ei = [&](int j, int x) { return j < nb ? std::sin(ang(j, x)) : 0.0; };
  auto Fr = [&](int j, int x) { return j < nb ? std::cos(ang(j, x)) : 0.0; };
  auto Fi = [&](int j, int x) { return j < nb ? -std::sin(ang(j, x)) : 0.0; };
  std::vector<unsigned char> img;
  switch (which) {
    case 0: {  // gemm 1, two A (rows x, K = j_x re | j_x im): [Er, -Ei] and [Ei, Er] at E[j_x][x]
      img.assign(2 * kTcImgY, 0);
      put_image(img.data(), n, 2 * nbp, [&](int x, int k) { return k < nbp ? Er(k, x) : -Ei(k - nbp, x); });
      put_image(img.data() + kTcImgY, n, 2 * nbp, [&](int x, int k) { return k < nbp ? Ei(k, x) : Er(k - nbp, x); });
      break;
    }
    case 1: {  // gemm 2, B (rows: re of y, then im of y; K = j_y re | j_y im) at E[j_y][y]
      img.assign((size_t)2 * n * 2 * nbp * 4, 0);
      put_image(img.data(), 2 * n, 2 * nbp, [&](int row, int k) {
        const int y = row % n;
        if (row < n) return k < nbp ? Er(k, y) : -Ei(k - nbp, y);
        return k < nbp ? Ei(k, y) : Er(k - nbp, y);
      });
      break;
    }
    case 2: {  // gemm 3, two A (rows k_y, padded to 128 with zeros; K = y re | y im) at F[k_y][y]
      img.assign(2 * kTcImgW, 0);
      put_image(img.data(), n, 2 * n, [&](int ky, int k) {
        if (ky >= nbp) return 0.0;
        return k < n ? Fr(ky, k) : -Fi(ky, k - n);
      });
      put_image(img.data() + kTcImgW, n, 2 * n, [&](int ky, int k) {
        if (ky >= nbp) return 0.0;
        return k < n ? Fi(ky, k) : Fr(ky, k - n);
      });
      break;
    }
    default: {  // gemm 4, B (rows: re of k_x, then im of k_x; K = x re | x im) at F[k_x][x]
      img.assign((size_t)2 * nbp * 2 * n * 4, 0);
      put_image(img.data(), 2 * nbp, 2 * n, [&](int row, int k) {
        const int kx = row % nbp;
        if (row < nbp) return k < n ? Fr(kx, k) : -Fi(kx, k - n);
        return k < n ? Fi(kx, k) : Fr(kx, k - n);
      });
      break;
    }
  }
  return img;
}

// ------------------------------------------------------------------ host: launches
template <int NA, int RB, int KR, int MODE>
static cudaError_t gemm_prepare() {
  return cudaFuncSetAttribute(tc_gemm_kernel<NA, RB, KR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)GemmShape<NA, RB, KR>::SMEM);
}

template <int NA, int RB, int KR, int MODE>
static cudaError_t gemm(const TcGemmArgs& g, int batch, cudaStream_t s) {
  tc_gemm_kernel<NA, RB, KR, MODE><<<batch, kTcThreads, GemmShape<NA, RB, KR>::SMEM, s>>>(g);
  return cudaGetLastError();
}

constexpr int kStencilSmem = 3 * kTcN * (kTcN + 1) * (int)sizeof(float);

cudaError_t prepare_tc() {
  cudaError_t e = gemm_prepare<2, kTcBand, 2 * kTcBand, kImage>();
  if (e == cudaSuccess) e = gemm_prepare<1, 2 * kTcN, 2 * kTcBand, kOT>();
  if (e == cudaSuccess) e = gemm_prepare<2, kTcN, 2 * kTcN, kImage>();
  if (e == cudaSuccess) e = gemm_prepare<1, 2 * kTcBand, 2 * kTcN, kG>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStencilSmem);
  return e;
}

cudaError_t launch_tc_tile(const TcArgs& a, cudaStream_t s) {
  const int K = a.K;
  tc_prep_kernel<<<K, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcGemmArgs g{};
  g.t = a;
  // gemm 1: Y'[x][j_y] = sum_jx E[j_x][x] X[j_y][j_x]        (A: E, two images; B: X)
  g.A = a.cA1; g.sA = 0; g.A2off = (long)kTcImgY;
  g.B = a.iX; g.sB = (long)kTcImgX;
  g.out = a.iY; g.sOut = (long)kTcImgY;
  if ((e = gemm<2, kTcBand, 2 * kTcBand, kImage>(g, K, s)) != cudaSuccess) return e;
  // gemm 2: O'[x][y] = sum_jy Y'[x][j_y] E[j_y][y]            (A: Y'; B: E, re and im rows)
  g.A = a.iY; g.sA = (long)kTcImgY; g.A2off = 0;
  g.B = a.cB2; g.sB = 0;
  g.out = nullptr; g.sOut = 0;
  if ((e = gemm<1, 2 * kTcN, 2 * kTcBand, kOT>(g, K, s)) != cudaSuccess) return e;
  tc_stencil_kernel<<<K, 1024, kStencilSmem, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // gemm 3: Z[k_y][x] = sum_y F[k_y][y] W'[x][y]              (A: F, two images; B: W')
  g.A = a.cA3; g.sA = 0; g.A2off = (long)kTcImgW;
  g.B = a.iW; g.sB = (long)kTcImgW;
  g.out = a.iZ; g.sOut = (long)kTcImgZ;
  if ((e = gemm<2, kTcN, 2 * kTcN, kImage>(g, K, s)) != cudaSuccess) return e;
  // gemm 4: G[k_y][k_x] = sum_x Z[k_y][x] F[k_x][x]           (A: Z; B: F, re and im rows)
  g.A = a.iZ; g.sA = (long)kTcImgZ; g.A2off = 0;
  g.B = a.cB4; g.sB = 0;
  g.out = nullptr; g.sOut = 0;
  return gemm<1, 2 * kTcBand, 2 * kTcN, kG>(g, K, s);
}

}  // namespace elf
