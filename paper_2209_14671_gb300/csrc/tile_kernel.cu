// Fused per-LED tile kernel: Eq. 1 forward field, Eq. 5 (or 4) residual, the
// normaliser of Eq. 12, W_n of Eq. 11 (or 10) and the F_B^H factor of Eq. 9.
//
// One LED = one thread-block cluster of CS CTAs.  The n x n tile never leaves
// on-chip memory:
//   A  each CTA inverse-transforms its share of the support band rows
//      (crop x pupil, zero outside the support) into its shared memory;
//   B  each CTA gathers, through distributed shared memory, the full columns it
//      owns (n/CS of them, plus one halo column on each side) and
//      inverse-transforms them, giving o_n on those columns;
//      then r = |o|^2 - I (coalesced reads of I), the forward-difference
//      gradient, the smoothed normaliser omega and W = o * nabla^T omega on the
//      owned columns, with the per-pixel cost accumulated in FP64;
//      then the forward column transforms of W;
//   C  each CTA gathers the band rows it owns from all CTAs' columns and
//      forward-transforms them, keeping the support pixels only (G_n).
// The (-1)^(x+y) factors realise ifftshift/fftshift for even n; the scale
// 1/(u^2 n^2) is applied to o and to G.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace elf {

constexpr int kTileThreads = 256;

template <int CS>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (CS > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

template <int CS, typename T>
__device__ __forceinline__ T* remote(T* p, int rank) {
  if constexpr (CS > 1) {
    return cg::this_cluster().map_shared_rank(p, rank);
  } else {
    return p;
  }
}

struct OmegaOut {
  float wx, wy, phi;
};

// Smoothed normaliser of Eq. 12 (reading A7) at pixel (y, x) from the residual r
// stored column-major in R (local column c = x - x0 + 1, pitch LD).
template <int NL, int LD>
__device__ __forceinline__ OmegaOut omega_at(const float* R, int y, int x, int c, float tau, int iso) {
  const float r0 = R[c * LD + y];
  const float dx = (x < NL - 1) ? R[(c + 1) * LD + y] - r0 : 0.f;
  const float dy = (y < NL - 1) ? R[c * LD + y + 1] - r0 : 0.f;
  OmegaOut o;
  if (iso) {
    const float nrm = sqrtf(dx * dx + dy * dy);
    const float den = fmaxf(nrm, tau);
    o.wx = dx / den;
    o.wy = dy / den;
    o.phi = (nrm >= tau) ? nrm : nrm * nrm / (2.f * tau) + 0.5f * tau;
  } else {
    const float ax = fabsf(dx), ay = fabsf(dy);
    o.wx = dx / fmaxf(ax, tau);
    o.wy = dy / fmaxf(ay, tau);
    o.phi = ((ax >= tau) ? ax : ax * ax / (2.f * tau) + 0.5f * tau) +
            ((ay >= tau) ? ay : ay * ay / (2.f * tau) + 0.5f * tau);
  }
  return o;
}

template <int NL, int CS>
__global__ void __launch_bounds__(kTileThreads) tile_kernel(const TileArgs a) {
  constexpr int NT = kTileThreads;
  constexpr int TL = FftTeam<NL>::TL;
  constexpr int NTEAM = NT / TL;
  constexpr int CW = NL / CS;     // owned columns
  constexpr int WC = CW + 2;      // with one halo column per side
  constexpr int LD = NL + 1;      // column pitch (padding against bank conflicts)

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* A1 = tw + NL;
  float2* OC = A1 + a.rowsA * NL;
  float* R = reinterpret_cast<float*>(OC + WC * LD);
  double* red = reinterpret_cast<double*>(R + ((WC * LD + 1) & ~1));

  const int tid = threadIdx.x;
  int crank = 0;
  if constexpr (CS > 1) crank = (int)cg::this_cluster().block_rank();
  const int led = blockIdx.x / CS;
  const int lane = tid % TL;
  const int team = tid / TL;

  for (int i = tid; i < NL; i += NT) tw[i] = a.tw[i];
  __syncthreads();

  const int2 org = a.origin[led];
  const int b0 = crank * a.rowsA;
  const int nrows = max(0, min(a.nb - b0, a.rowsA));

  // ---- A: inverse row transforms of this CTA's band rows
  for (int base = 0; base < a.rowsA; base += NTEAM) {
    const int lb = base + team;
    const bool act = lb < nrows;
    float2* row = A1 + (act ? lb : 0) * NL;
    if (act) {
      const int y = a.Blo + b0 + lb;
      const int xs = a.row_xs[y], cnt = a.row_cnt[y];
      const float2* prow = a.psi + (size_t)(org.x + y) * a.N + org.y;
      for (int x = lane; x < NL; x += TL) {
        float2 v = make_float2(0.f, 0.f);
        if ((unsigned)(x - xs) < (unsigned)cnt) v = cmul(a.pupil[y * NL + x], prow[x]);
        row[x] = v;
      }
    }
    __syncwarp();
    team_fft<NL, true>(row, tw, lane, act);
  }
  cluster_barrier<CS>();

  // ---- B: inverse column transforms of the owned + halo columns
  const int x0 = crank * CW;
  for (int base = 0; base < WC; base += NTEAM) {
    const int lc = base + team;
    const int x = x0 - 1 + lc;
    const bool act = (lc < WC) && x >= 0 && x < NL;
    float2* col = OC + (act ? lc : 0) * LD;
    if (act) {
      for (int y = lane; y < NL; y += TL) {
        const int b = y - a.Blo;
        float2 v = make_float2(0.f, 0.f);
        if ((unsigned)b < (unsigned)a.nb) {
          const int own = b / a.rowsA;
          const float2* src = remote<CS>(A1, own);
          v = src[(b - own * a.rowsA) * NL + x];
        }
        col[y] = v;
      }
    }
    __syncwarp();
    team_fft<NL, true>(col, tw, lane, act);
  }
  __syncthreads();

  // o = (-1)^(x+y) scale * IDFT, and the residual r (coalesced reads of I)
  const size_t img = (size_t)led * NL * NL;
  for (int p = tid; p < NL * WC; p += NT) {
    const int y = p / WC;
    const int lc = p - y * WC;
    const int x = x0 - 1 + lc;
    if (x < 0 || x >= NL) continue;
    float2 o = OC[lc * LD + y];
    const float sg = ((x + y) & 1) ? -a.scale : a.scale;
    o.x *= sg;
    o.y *= sg;
    OC[lc * LD + y] = o;
    const float m2 = cabs2(o);
    if (a.mode == 1) {
      if (lc >= 1 && lc <= CW) a.I_out[img + (size_t)y * NL + x] = m2;
      continue;
    }
    const float meas = a.meas[img + (size_t)y * NL + x];
    R[lc * LD + y] = (a.fidelity == 0) ? (m2 - meas) : (sqrtf(m2) - sqrtf(fmaxf(meas, 0.f)));
  }
  if (a.mode == 1) {
    cluster_barrier<CS>();  // peers may still be reading this CTA's A1
    return;
  }
  __syncthreads();

  // W = o * nabla^T omega (Eq. 11) or o / (2 max(|o|, eta)) * nabla^T omega (Eq. 10),
  // times (-1)^(x+y) for the forward shift; cost phi summed over owned pixels.
  double acc = 0.0;
  for (int p = tid; p < NL * CW; p += NT) {
    const int cw = p / NL;
    const int y = p - cw * NL;
    const int c = cw + 1;
    const int x = x0 + cw;
    const OmegaOut w0 = omega_at<NL, LD>(R, y, x, c, a.tau, a.iso);
    float w = -w0.wx - w0.wy;
    if (x >= 1) w += omega_at<NL, LD>(R, y, x - 1, c - 1, a.tau, a.iso).wx;
    if (y >= 1) w += omega_at<NL, LD>(R, y - 1, x, c, a.tau, a.iso).wy;
    acc += (double)w0.phi;
    float2 o = OC[c * LD + y];
    float f = w;
    if (a.fidelity != 0) f = w / (2.f * fmaxf(sqrtf(cabs2(o)), a.eta));
    if ((x + y) & 1) f = -f;
    OC[c * LD + y] = cscale(o, f);
  }
  // block reduction of the FP64 cost partial (fixed order)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < NT / 32; ++i) s += red[i];
    a.costpart[led * CS + crank] = s;
  }

  // forward column transforms of the owned columns
  for (int base = 0; base < CW; base += NTEAM) {
    const int cw = base + team;
    const bool act = cw < CW;
    team_fft<NL, false>(OC + (act ? cw + 1 : 1) * LD, tw, lane, act);
  }
  cluster_barrier<CS>();

  // ---- C: forward row transforms of this CTA's band rows; keep the support
  for (int base = 0; base < a.rowsA; base += NTEAM) {
    const int lb = base + team;
    const bool act = lb < nrows;
    float2* row = A1 + (act ? lb : 0) * NL;
    const int ky = a.Blo + b0 + (act ? lb : 0);
    if (act) {
      for (int x = lane; x < NL; x += TL) {
        const int own = x / CW;
        const float2* src = remote<CS>(OC, own);
        row[x] = src[(x - own * CW + 1) * LD + ky];
      }
    }
    __syncwarp();
    team_fft<NL, false>(row, tw, lane, act);
    if (act) {
      const int xs = a.row_xs[ky], cnt = a.row_cnt[ky];
      float2* dst = a.G + (size_t)led * a.S + a.row_off[ky];
      for (int i = lane; i < cnt; i += TL) dst[i] = cscale(row[xs + i], a.scale);
    }
  }
  cluster_barrier<CS>();  // keep this CTA's columns alive until every peer has read them
}

int tile_cluster_size(int n) {
  switch (n) {
    case 256: return 8;
    case 128: return 4;
    default: return 1;
  }
}

size_t tile_smem_bytes(int n, int cs, int rowsA) {
  const size_t wc = n / cs + 2, ld = n + 1;
  return 8 * ((size_t)n + (size_t)rowsA * n + wc * ld) + 4 * ((wc * ld + 1) & ~(size_t)1) +
         8 * (kTileThreads / 32);
}

template <int NL, int CS>
static cudaError_t launch_tile_t(const TileArgs& a, cudaStream_t s) {
  const size_t smem = tile_smem_bytes(NL, CS, a.rowsA);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.K * CS);
  cfg.blockDim = dim3(kTileThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (CS > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS>, a);
}

template <int NL, int CS>
static cudaError_t prepare_tile_t(int rowsA) {
  static int configured = 0;  // largest dynamic shared memory size set so far
  const int smem = (int)tile_smem_bytes(NL, CS, rowsA);
  if (smem <= configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(tile_kernel<NL, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) configured = smem;
  return e;
}

cudaError_t prepare_tile(int n, int rowsA) {
  switch (n) {
    case 16: return prepare_tile_t<16, 1>(rowsA);
    case 32: return prepare_tile_t<32, 1>(rowsA);
    case 64: return prepare_tile_t<64, 1>(rowsA);
    case 128: return prepare_tile_t<128, 4>(rowsA);
    case 256: return prepare_tile_t<256, 8>(rowsA);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile(const TileArgs& a, int n, cudaStream_t s) {
  switch (n) {
    case 16: return launch_tile_t<16, 1>(a, s);
    case 32: return launch_tile_t<32, 1>(a, s);
    case 64: return launch_tile_t<64, 1>(a, s);
    case 128: return launch_tile_t<128, 4>(a, s);
    case 256: return launch_tile_t<256, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace elf
