// Per-LED tile work of the fidelity gradient (Eqs. 1, 5 or 4, 12, 11 or 10 and the F_B^H factor
// of Eq. 9) as three cluster-free kernels that pass the pupil-support band of every LED's tile
// through global memory (L2-resident at the sizes used: 2 x K x nb x n complex):
//
//   rows_inv   one FFT team per (LED, band row): crop x pupil (zero off the support) loaded
//              straight into the transform's registers, the inverse row transform, the row
//              written to band_in[LED][b][0..n);
//   cols       one CTA per (LED, strip of CW columns): the strip's band columns plus one halo
//              column per side are read from band_in, inverse-transformed along the columns
//              (only the band rows are non-zero), giving o_n on the strip; then the residual,
//              the smoothed normaliser of Eq. 12 and W = o * nabla^T omega in one register-carried
//              pass per row strip, with the cost summed per warp as an unevaluated (hi, lo) float
//              pair; then the forward column transforms of the owned columns, whose band rows go
//              to band_out[LED][b][strip];
//   rows_fwd   one FFT team per (LED, band row): the forward row transform of band_out, the
//              support pixels scaled into G.
//
// Every CTA is independent: no clusters, so every SM takes work, and two column CTAs (about
// 113 KB of shared memory each at n = 256) share an SM, overlapping each other's barriers.
// The (-1)^(x+y) factors of ifftshift / fftshift cancel in W and are never applied; the scale
// 1/(u^2 n^2) is applied to o (through |o|) and to G.
#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace elf {

namespace {

constexpr int kRowThreads = 256;

template <int NL> struct SplitCfg {
  static constexpr int CW = NL < 32 ? NL : 32;  // owned columns per column CTA
  static constexpr int NT = NL >= 256 ? 288 : NL >= 64 ? 288 : 256;
  static constexpr int MINB = 2;               // column CTAs per SM the registers are bounded for
};

// Row pitch (in float2) of the column buffer: at least the CW + 2 owned and halo columns, chosen
// so that the strided column transforms of one half-warp fall in distinct banks.
__host__ __device__ constexpr int split_pitch(int n) {
  return n == 256 ? 35 : n == 128 ? 34 : n == 64 ? 34 : n == 32 ? 36 : 20;
}

__host__ __device__ constexpr int pow2_floor_w(int w) { return w >= 16 ? 16 : w >= 8 ? 8 : w >= 4 ? 4 : w >= 2 ? 2 : 1; }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------ rows: inverse (stage A)
template <int NL>
__global__ void __launch_bounds__(kRowThreads) rows_inv_kernel(const TileArgs a, float2* __restrict__ band) {
  using T = FftTeam<NL>;
  constexpr int TL = T::TL, NTEAM = kRowThreads / TL, RP = T::PADDED, PL = T::P, Q = T::Q;
  __shared__ __align__(16) float2 tw[NL];
  __shared__ __align__(16) float2 rows[NTEAM * RP];
  pdl_launch_dependents();
  const int tid = threadIdx.x, lane = tid % TL, team = tid / TL;
  for (int i = tid; i < NL; i += kRowThreads) tw[i] = a.tw[i];
  const int nb = a.nb, nl = a.nled > 0 ? a.nled : a.K;
  const int g = blockIdx.x * NTEAM + team;
  const bool act = g < nl * nb;
  const int led = a.led0 + (act ? g / nb : 0), b = act ? g % nb : 0;
  const int y = a.Blo + b;
  float2 v[PL];
  if (act) {
    const int2 org = a.origin[led];
    const int xs = a.row_xs[y], cnt = a.row_cnt[y];
    const float2* prow = a.psi + (size_t)(org.x + y) * a.N + org.y;
    const float2* pp = a.pupil + (size_t)y * NL;
    float2 pv[PL];
#pragma unroll
    for (int j = 0; j < PL; ++j) {
      const int x = lane + TL * j;
      const bool in = (unsigned)(x - xs) < (unsigned)cnt;
      pv[j] = in ? pp[x] : make_float2(0.f, 0.f);
      v[j] = in ? prow[x] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < PL; ++j) v[j] = cscale(cmul(pv[j], v[j]), a.scale);  // scale folded in (see load_o)
  }
  __syncthreads();  // twiddles
  team_fft_core<NL, true>(v, rows + team * RP, tw, lane, act);
  if (act) {
    float2* dst = band + ((size_t)(led - a.led0) * nb + b) * NL;
#pragma unroll
    for (int m = 0; m < PL / Q; ++m)
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) dst[lane + Q * m + PL * k2] = v[m * Q + k2];
  }
}

// ------------------------------------------------------------------ rows: forward (stage C)
template <int NL>
__global__ void __launch_bounds__(kRowThreads) rows_fwd_kernel(const TileArgs a, const float2* __restrict__ band) {
  using T = FftTeam<NL>;
  constexpr int TL = T::TL, NTEAM = kRowThreads / TL, RP = T::PADDED, PL = T::P, Q = T::Q;
  __shared__ __align__(16) float2 tw[NL];
  __shared__ __align__(16) float2 rows[NTEAM * RP];
  const int tid = threadIdx.x, lane = tid % TL, team = tid / TL;
  for (int i = tid; i < NL; i += kRowThreads) tw[i] = a.tw[i];
  const int nb = a.nb, nl = a.nled > 0 ? a.nled : a.K;
  const int g = blockIdx.x * NTEAM + team;
  const bool act = g < nl * nb;
  const int li = act ? g / nb : 0, b = act ? g % nb : 0;
  pdl_wait();  // band_out of the column kernel
  float2 v[PL];
  if (act) {
    const float2* src = band + ((size_t)li * nb + b) * NL;
#pragma unroll
    for (int j = 0; j < PL; ++j) v[j] = src[lane + Q * j];
  }
  __syncthreads();  // twiddles
  team_fft_core<NL, false>(v, rows + team * RP, tw, lane, act);
  if (act) {
    const int ky = a.Blo + b;
    const int xs = a.row_xs[ky], cnt = a.row_cnt[ky];
    float2* dst = a.G + (size_t)(a.led0 + li) * a.S + a.row_off[ky];
#pragma unroll
    for (int m = 0; m < PL / Q; ++m)
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        const int d = lane + Q * m + PL * k2 - xs;
        if ((unsigned)d < (unsigned)cnt) dst[d] = cscale(v[m * Q + k2], a.scale);
      }
  }
}

// ------------------------------------------------------------------ columns + stencil (stage B)
struct Om {
  float wx, wy, phi;
};

template <int NL>
size_t cols_smem_bytes() {
  constexpr int CW = SplitCfg<NL>::CW, NT = SplitCfg<NL>::NT;
  return 4 * (size_t)NL * CW + 4 * 2 * (size_t)NL + 8 * (size_t)NL +
         8 * (size_t)FftTeam<NL>::PADDED * split_pitch(NL) + 4 * 2 * (size_t)NL + 8 * (size_t)(NT / 32);
}

// FID: 0 = intensity (Eq. 5), 1 = amplitude (Eq. 4; meas holds sqrt(max(I, 0))), 2 = a Sec. 6.3 map
// (power or log by a.fidelity; meas holds g(max(I, 0))); ISO: isotropic (1) or anisotropic (0)
// normaliser of Eq. 12.
template <int NL, int FID, int ISO>
__global__ void __launch_bounds__(SplitCfg<NL>::NT, SplitCfg<NL>::MINB)
    cols_kernel(const TileArgs a, const float2* __restrict__ band_in, float2* __restrict__ band_out) {
  constexpr int CW = SplitCfg<NL>::CW, NT = SplitCfg<NL>::NT, NW = NT / 32;
  constexpr int STRIPS = NL / CW;
  constexpr int TL = FftTeam<NL>::TL, NTEAM = NT / TL;
  constexpr int WC = CW + 2;
  constexpr int RP = FftTeam<NL>::PADDED;
  constexpr int PO = split_pitch(NL);
  static_assert(PO >= WC, "rows of the column buffer hold the owned and halo columns");
  static_assert(CW <= 32, "one warp spans the owned columns");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Itile = reinterpret_cast<float*>(smem_raw);  // NL x CW measured values (row-major)
  float* Ihalo = Itile + NL * CW;                      // 2 x NL: the halo columns x0 - 1, x0 + CW
  float2* tw = reinterpret_cast<float2*>(Ihalo + 2 * NL);
  float2* OC = tw + NL;                                // RP rows of PO: row pidx(y), column 1 + x - x0
  float* Hx = reinterpret_cast<float*>(OC + RP * PO);  // 2 x NL: r at x0 + CW, omega_x at x0 - 1
  float2* cpair = reinterpret_cast<float2*>(Hx + 2 * NL);

  const int tid = threadIdx.x, warp = tid >> 5, wl = tid & 31;
  const int lane = tid % TL, team = tid / TL;
  const int li = blockIdx.x / STRIPS, strip = blockIdx.x - li * STRIPS;
  const int led = a.led0 + li;
  const int x0 = strip * CW;
  const int nb = a.nb, Blo = a.Blo;
  const size_t img = (size_t)led * NL * NL;

  pdl_launch_dependents();
  // group 0: twiddles and the measured values (independent of the inverse row kernel, issued before
  // waiting for it); group 1: the band columns of the strip (+ halo) it wrote
  for (int i = tid; i < NL / 2; i += NT) cp_async16(tw + 2 * i, a.tw + 2 * i);
  {
    constexpr int CH = CW / 4;  // 16-byte chunks per row
    for (int i = tid; i < NL * CH; i += NT) {
      const int y = i / CH, k = i - y * CH;
      cp_async16(Itile + y * CW + 4 * k, a.meas + img + (size_t)y * NL + x0 + 4 * k);
    }
    for (int i = tid; i < 2 * NL; i += NT) {
      const int side = i / NL, y = i - side * NL;
      const int x = side ? x0 + CW : x0 - 1;
      if (x >= 0 && x < NL) cp_async4(Ihalo + i, a.meas + img + (size_t)y * NL + x);
    }
  }
  cp_commit();
  pdl_wait();  // band_in of the inverse row kernel
  {
    const float2* src = band_in + (size_t)li * nb * NL;
    for (int i = tid; i < nb * WC; i += NT) {
      const int b = i / WC, c = i - b * WC;
      const int x = x0 - 1 + c;
      if (x >= 0 && x < NL) cp_async8(OC + FftTeam<NL>::pidx(Blo + b) * PO + c, src + (size_t)b * NL + x);
    }
  }
  cp_commit();
  cp_wait<0>();
  __syncthreads();

  // inverse column transforms of the owned and halo columns (band rows only are non-zero)
  for (int base = 0; base < WC; base += NTEAM) {
    const int lc = base + team;
    const int x = x0 - 1 + lc;
    const bool act = (lc < WC) && x >= 0 && x < NL;
    team_fft<NL, true, PO>(OC + (act ? lc : 0), tw, lane, act, Blo, nb);
  }
  __syncthreads();

  // o~ = scale * IDFT without the (-1)^(x+y) factor: |o~| = |o| and (-1)^(x+y) o w = o~ w.  The scale,
  // 1 / (u^2 n^2), a power of two, was applied to the row kernel's input; a power of two commutes
  // exactly with every rounding of the transform, so o~ is bitwise what scaling here would give
  auto load_o = [&](int y, int c) -> float2 { return OC[FftTeam<NL>::pidx(y) * PO + c]; };
  const bool gpow = a.fidelity == 2;
  const float eta2 = a.eta * a.eta;
  auto resid_sl = [&](float2 o, float meas, float& sl) -> float {
    const float m2 = cabs2(o);
    if constexpr (FID == 0) {
      return m2 - meas;
    } else if constexpr (FID == 1) {
      return sqrtf(m2) - meas;
    } else {
      if (gpow) {
        const float p = powf(fmaxf(m2, eta2), a.gexp - 1.f);
        sl = a.gexp * p;
        return m2 * p - meas;
      }
      sl = 1.f / (m2 + 1.f);
      return log1pf(m2) - meas;
    }
  };
  auto resid = [&](float2 o, float meas) -> float {
    float sl;
    return resid_sl(o, meas, sl);
  };

  float acc = 0.f;
  {
    constexpr int SW = pow2_floor_w(NW);  // strip warps
    constexpr int RPW = NL / SW;          // rows per strip
    static_assert(RPW * SW == NL, "strips tile the rows");
    const float tau = a.tau, tau2 = fmaxf(a.tau * a.tau, 1e-36f), hit = (a.tau > 0.f) ? 0.5f / a.tau : 0.f;
    const bool on = wl < CW;
    const int cc = on ? wl : 0;
    const int c = cc + 1, x = x0 + cc;
    const bool has_left = x0 >= 1, has_right = x0 + CW < NL;
    const bool strip_w = warp < SW;
    const int ybeg = strip_w ? warp * RPW : 0, yend = strip_w ? ybeg + RPW : 0;
    auto r_own = [&](int y) { return resid(load_o(y, c), Itile[y * CW + cc]); };
    auto r_left = [&](int y) { return resid(load_o(y, 0), Ihalo[y]); };
    auto r_right = [&](int y) { return resid(load_o(y, CW + 1), Ihalo[NL + y]); };
    auto huber2 = [&](float dx, float dy) -> Om {
      Om o;
      if constexpr (ISO != 0) {
        const float ss = dx * dx + dy * dy;
        const float inv = rsqrtf(fmaxf(ss, tau2));
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
    };
    // halo tables: r at the right halo column and omega_x at the left halo column, every row
    for (int y = tid; y < NL; y += NT) {
      Hx[y] = has_right ? r_right(y) : 0.f;
      float wl_x = 0.f;
      if (has_left) {
        const float rl = r_left(y);
        const float dxl = resid(load_o(y, 1), Itile[y * CW]) - rl;
        const float dyl = (y < NL - 1) ? r_left(y + 1) - rl : 0.f;
        wl_x = huber2(dxl, dyl).wx;
      }
      Hx[NL + y] = wl_x;
    }
    // rows outside the strip, read before the barrier (their owners overwrite them with W)
    const float r_above = (strip_w && ybeg >= 1) ? r_own(ybeg - 1) : 0.f;
    const float r_below = (strip_w && yend < NL) ? r_own(yend) : 0.f;
    __syncthreads();
    if (strip_w) {
      float2 o_cur = load_o(ybeg, c);
      float sl_cur = 0.f, sl_nxt = 0.f;
      float r_cur = resid_sl(o_cur, Itile[ybeg * CW + cc], sl_cur);
      float wy_prev = 0.f;  // omega_y of the row above the strip (0 above the first row)
      if (ybeg >= 1) {
        float rr = __shfl_down_sync(0xffffffffu, r_above, 1);
        if (wl == CW - 1) rr = Hx[ybeg - 1];
        const float dx = (x < NL - 1) ? rr - r_above : 0.f;
        wy_prev = huber2(dx, r_cur - r_above).wy;
      }
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const int y = ybeg + i;
        float2 o_nxt;
        float r_nxt;
        if (i + 1 < RPW) {
          o_nxt = load_o(y + 1, c);
          r_nxt = resid_sl(o_nxt, Itile[(y + 1) * CW + cc], sl_nxt);
        } else {
          o_nxt = o_cur;
          r_nxt = (yend < NL) ? r_below : r_cur;
        }
        float rr = __shfl_down_sync(0xffffffffu, r_cur, 1);
        if (wl == CW - 1) rr = Hx[y];
        const float dx = (x < NL - 1) ? rr - r_cur : 0.f;
        const float dy = r_nxt - r_cur;
        const Om w0 = huber2(dx, dy);
        float wx_left = __shfl_up_sync(0xffffffffu, w0.wx, 1);
        if (wl == 0) wx_left = Hx[NL + y];  // 0 left of the image
        if (on) {
          float w = -w0.wx - w0.wy;
          w += wx_left;
          w += wy_prev;
          acc += w0.phi;
          float f = w;
          if constexpr (FID == 1) f = w * (0.5f * rsqrtf(fmaxf(cabs2(o_cur), eta2)));  // 1 / (2 max(|o|, eta))
          if constexpr (FID == 2) f = w * sl_cur;
          OC[FftTeam<NL>::pidx(y) * PO + c] = cscale(o_cur, f);
        }
        wy_prev = w0.wy;
        sl_cur = sl_nxt;
        o_cur = o_nxt;
        r_cur = r_nxt;
      }
    }
  }
  {
    const FF wsum = warp_sum_ff(FF{acc, 0.f});
    if (wl == 0) cpair[warp] = make_float2(wsum.hi, wsum.lo);
  }
  __syncthreads();  // W complete in every owned column
  // forward column transforms of the owned columns; only the band rows of the output are kept
  for (int base = 0; base < CW; base += NTEAM) {
    const int cw = base + team;
    const bool act = cw < CW;
    float2* col = OC + (act ? cw + 1 : 1);
    constexpr int PL = FftTeam<NL>::P, Q = FftTeam<NL>::Q;
    float2 v[PL];
    if (act) {
#pragma unroll
      for (int j = 0; j < PL; ++j) v[j] = col[(lane + (Q + 1) * j) * PO];
    }
    team_fft_core<NL, false, PO>(v, col, tw, lane, act);
    if (act) {
#pragma unroll
      for (int m = 0; m < PL / Q; ++m)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int k = lane + Q * m + PL * k2;
          if ((unsigned)(k - Blo) < (unsigned)nb) col[FftTeam<NL>::pidx(k) * PO] = v[m * Q + k2];
        }
    }
  }
  __syncthreads();
  {
    float2* dst = band_out + (size_t)li * nb * NL + x0;
    for (int i = tid; i < nb * CW; i += NT) {
      const int b = i / CW, cc = i - b * CW;
      dst[(size_t)b * NL + cc] = OC[FftTeam<NL>::pidx(Blo + b) * PO + cc + 1];
    }
  }
  if (tid == 0) {  // the warps' cost pairs in warp order: one pair per (LED, strip)
    FF s = {cpair[0].x, cpair[0].y};
    for (int w = 1; w < NW; ++w) s = ff_add(s, FF{cpair[w].x, cpair[w].y});
    a.cost_ff[(size_t)led * STRIPS + strip] = make_float2(s.hi, s.lo);
  }
}

template <int NL>
cudaError_t launch_split_t(const TileArgs& a, float2* band_in, float2* band_out, cudaStream_t s) {
  using T = FftTeam<NL>;
  constexpr int NTEAM = kRowThreads / T::TL;
  constexpr int CW = SplitCfg<NL>::CW, NT = SplitCfg<NL>::NT;
  const int nl = a.nled > 0 ? a.nled : a.K;
  if (nl <= 0 || a.nb <= 0) return cudaSuccess;
  const int rows = nl * a.nb;
  rows_inv_kernel<NL><<<(rows + NTEAM - 1) / NTEAM, kRowThreads, 0, s>>>(a, band_in);
  const size_t smem = cols_smem_bytes<NL>();
  const dim3 grid(nl * (NL / CW));
  const int fid = (a.fidelity >= 2) ? 2 : a.fidelity;
  const float2* bin = band_in;
  cudaError_t e;
  switch (2 * fid + (a.iso ? 1 : 0)) {
    case 0: e = launch_dependent(cols_kernel<NL, 0, 0>, grid, dim3(NT), smem, s, a, bin, band_out); break;
    case 1: e = launch_dependent(cols_kernel<NL, 0, 1>, grid, dim3(NT), smem, s, a, bin, band_out); break;
    case 2: e = launch_dependent(cols_kernel<NL, 1, 0>, grid, dim3(NT), smem, s, a, bin, band_out); break;
    case 3: e = launch_dependent(cols_kernel<NL, 1, 1>, grid, dim3(NT), smem, s, a, bin, band_out); break;
    case 4: e = launch_dependent(cols_kernel<NL, 2, 0>, grid, dim3(NT), smem, s, a, bin, band_out); break;
    default: e = launch_dependent(cols_kernel<NL, 2, 1>, grid, dim3(NT), smem, s, a, bin, band_out); break;
  }
  if (e != cudaSuccess) return e;
  const float2* bout = band_out;
  e = launch_dependent(rows_fwd_kernel<NL>, dim3((rows + NTEAM - 1) / NTEAM), dim3(kRowThreads), 0, s, a, bout);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NL>
cudaError_t prepare_split_t() {
  const int smem = (int)cols_smem_bytes<NL>();
  cudaError_t e = cudaSuccess;
  for (auto k : {cols_kernel<NL, 0, 0>, cols_kernel<NL, 0, 1>, cols_kernel<NL, 1, 0>, cols_kernel<NL, 1, 1>,
                 cols_kernel<NL, 2, 0>, cols_kernel<NL, 2, 1>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

}  // namespace

bool tile_split_selected(int n, int mux, int tile_dft, int tile_path) {
  if (mux > 1 || tile_dft) return false;
  if (tile_path == 2) return true;
  if (tile_path == 1) return false;
  // automatic: measured on GB300 with 225 LEDs, an iteration takes 0.166 against 0.233 ms at n = 256
  // and 0.054 against 0.059 ms at n = 128 (8-iteration graphs) with the split kernels; at n = 64 the
  // two are within 2 %, and the cluster kernel is kept there
  return n >= 128;
}

cudaError_t prepare_tile_split(int n) {
  switch (n) {
    case 16: return prepare_split_t<16>();
    case 32: return prepare_split_t<32>();
    case 64: return prepare_split_t<64>();
    case 128: return prepare_split_t<128>();
    case 256: return prepare_split_t<256>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_split(const TileArgs& a, int n, float2* band_in, float2* band_out, cudaStream_t s) {
  if (a.mode != 0) return cudaErrorInvalidValue;  // gradient mode only
  switch (n) {
    case 16: return launch_split_t<16>(a, band_in, band_out, s);
    case 32: return launch_split_t<32>(a, band_in, band_out, s);
    case 64: return launch_split_t<64>(a, band_in, band_out, s);
    case 128: return launch_split_t<128>(a, band_in, band_out, s);
    case 256: return launch_split_t<256>(a, band_in, band_out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace elf
