// Fused per-LED tile kernel: Eq. 1 forward field, Eq. 5 (or 4) residual, the
// normaliser of Eq. 12, W_n of Eq. 11 (or 10) and the F_B^H factor of Eq. 9.
//
// One LED = one thread-block cluster of CS CTAs.  The n x n tile never leaves
// on-chip memory:
//   0  each CTA starts asynchronous copies (cp.async) of the twiddles and of its
//      columns of I_n, and arrives at the cluster barrier it waits on in stage A;
//   A  each CTA inverse-transforms its share of the support band rows
//      (crop x pupil, zero outside the support, loaded straight into the
//      transform's registers) and pushes the results from registers with
//      distributed-shared-memory stores into the rows of the CTA owning each
//      column (and of the neighbour that keeps it as a halo column): contiguous
//      remote stores only, no remote loads;
//   B  each CTA inverse-transforms the full columns it owns (n/CS of them, plus
//      one halo column on each side), giving o_n on those columns;
//      then r = |o|^2 - I, the forward-difference gradient, the smoothed
//      normaliser omega and W = o * nabla^T omega on the owned columns, with the
//      per-pixel cost summed per warp as an unevaluated (hi, lo) float pair;
//      then the forward column transforms of W, whose band rows are pushed to
//      the CTAs owning those rows;
//   C  each CTA forward-transforms its band rows and writes the support pixels
//      (G_n) from the transform's registers.
// The column buffer OC is row-major (row pidx(y), one column per owned or halo x)
// with a pitch that keeps the strided column transforms free of bank conflicts.
// The (-1)^(x+y) factors realise ifftshift/fftshift for even n; the scale
// 1/(u^2 n^2) is applied to o and to G.
#include <cooperative_groups.h>

#include "dsmem.cuh"
#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace cg = cooperative_groups;

namespace elf {

// Tile configuration per image side n: cluster size CS and threads per CTA NT.
// A CTA owns n/CS = 32 columns and transforms 34 (one halo column per side), so NT
// holds at least 34 FFT teams and every column pass is a single round:
//   n = 256: 8 CTAs of 544 threads (34 teams of 16 lanes; ~137 KB shared memory, one per SM)
//   n = 128: 4 CTAs of 288 threads (36 teams of 8; ~64 KB), n = 64: 2 CTAs of 288 (~36 KB)
template <int NL> struct TileCfg { static constexpr int CS = 1, NT = 256; };
template <> struct TileCfg<64> { static constexpr int CS = 2, NT = 288; };
template <> struct TileCfg<128> { static constexpr int CS = 4, NT = 288; };
template <> struct TileCfg<256> { static constexpr int CS = 8, NT = 544; };

// Row pitch (in float2) of the per-CTA column buffer: at least the 34 (or n + 2) owned and
// halo columns, and chosen so that the column transforms' strided accesses by the teams
// of one half-warp fall in distinct banks (odd for 16-lane teams, 2 mod 16 for 8-lane
// teams, 4 mod 16 for 4-lane teams).
__host__ __device__ constexpr int oc_pitch(int n) {
  return n == 256 ? 35 : n == 128 ? 34 : n == 64 ? 34 : n == 32 ? 36 : 20;
}

// largest power of two <= w (the warps that walk row strips in the stencil pass)
__host__ __device__ constexpr int pow2_floor(int w) { return w >= 16 ? 16 : w >= 8 ? 8 : w >= 4 ? 4 : w >= 2 ? 2 : 1; }


// The smoothed normaliser of Eq. 12 (reading A7) at one pixel: omega = d / max(|d|, tau),
// phi = |d| (|d| >= tau) or |d|^2/(2 tau) + tau/2 (per component when anisotropic).
struct OmegaOut {
  float wx, wy, phi;
};

// FID: 0 = intensity fidelity (Eq. 5), 1 = amplitude (Eq. 4; meas holds sqrt(max(I, 0))), 2 = a scaling
// map of Sec. 6.3 (power or log, chosen at run time by a.fidelity = 2 or 3; meas holds g(max(I, 0))); ISO: 1 = isotropic
// normaliser, 0 = anisotropic (Eq. 12).  Compile-time, so the per-pixel loops carry no untaken branch
// work in the two forms of the paper's Eqs. 4-5.
template <int NL, int CS, int NT, int FID, int ISO>
__global__ void __launch_bounds__(NT) tile_kernel(const TileArgs a) {
  constexpr int NW = NT / 32;
  constexpr int TL = FftTeam<NL>::TL;
  constexpr int NTEAM = NT / TL;
  constexpr int CW = NL / CS;     // owned columns
  constexpr int WC = CW + 2;      // with one halo column per side
  constexpr int RP = FftTeam<NL>::PADDED;  // FFT buffer length (padded layout)
  constexpr int PO = oc_pitch(NL);          // row pitch of OC (conflict-free column transforms)
  static_assert(PO >= WC, "OC rows hold the owned and halo columns");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Itile = reinterpret_cast<float*>(smem_raw);      // NL x CW measured intensities (row-major)
  float* Ihalo = Itile + NL * CW;                          // 2 x NL: the halo columns x0-1, x0+CW
  float2* tw = reinterpret_cast<float2*>(Ihalo + 2 * NL);
  float2* A1 = tw + NL;                                   // rowsA band rows of pitch RP
  float2* OC = A1 + a.rowsA * RP;                         // RP rows of PO: row pidx(y), column 1 + x - x0
  float* Hx = reinterpret_cast<float*>(OC + RP * PO);     // 2 x NL: r at x0+CW, omega_x at x0-1

  const int tid = threadIdx.x;
  const int warp = tid >> 5, wl = tid & 31;
  int crank = 0;
  if constexpr (CS > 1) crank = (int)cg::this_cluster().block_rank();
  const int led = a.led0 + (int)blockIdx.x / CS;
  const int lane = tid % TL;
  const int team = tid / TL;
  const int x0 = crank * CW;
  const size_t img = (size_t)led * NL * NL;
  // mode 2 (multiplexed images) reads the factor f of the LED's image j = led / M in place of I
  const size_t meas_img = (size_t)(a.mode == 2 ? led / a.mux : led) * NL * NL;
  const bool has_meas = a.mode != 1;

  // twiddles (group 0) and this CTA's columns of I_n (group 1, overlapping stages A and B)
  // arrive by cp.async in 16-byte chunks
  {
    const unsigned tbase = (unsigned)__cvta_generic_to_shared(tw);
    for (int i = tid; i < NL / 2; i += NT)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tbase + 16u * i), "l"(a.tw + 2 * i)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (has_meas) {
    constexpr int CH = CW / 4;  // 16-byte chunks per row
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(Itile);
    for (int i = tid; i < NL * CH; i += NT) {
      const int y = i / CH, k = i - y * CH;
      const float* src = a.meas + meas_img + (size_t)y * NL + x0 + 4 * k;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sbase + 4u * (y * CW + 4 * k)), "l"(src)
                   : "memory");
    }
    for (int i = tid; i < (a.mode == 0 ? 2 * NL : 0); i += NT) {  // halo columns: mode 0 only
      const int side = i / NL, y = i - side * NL;
      const int x = side ? x0 + CW : x0 - 1;
      if (x < 0 || x >= NL) continue;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sbase + 4u * (NL * CW + i)),
                   "l"(a.meas + img + (size_t)y * NL + x)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  const int b0 = crank * a.rowsA;
  const int nrows = max(0, min(a.nb - b0, a.rowsA));
  // mbarriers of the two exchanges into this CTA: [0] the stage A rows of its owned and halo
  // columns (every band row, CW columns plus a halo column on each inner side), [1] its stage C
  // rows (all n columns of each of its band rows)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Hx + 2 * NL);
  if constexpr (CS > 1) {
    if (tid == 0) {
      const int cols = CW + (crank > 0 ? 1 : 0) + (crank < CS - 1 ? 1 : 0);
      mbar_init_expect(&mbar[0], (uint32_t)(a.nb * cols * 8));
      mbar_init_expect(&mbar[1], (uint32_t)(nrows * NL * 8));
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
  }
  // Every CTA of the cluster must be running, with its mbarriers initialised, before the first
  // remote store: arrive now, wait just before the stage A pushes, so that the barrier's latency
  // overlaps the crop loads and the first transforms.
  cluster_arrive<CS>();

  const int2 org = a.origin[led];

  // ---- A: inverse row transforms of this CTA's band rows, pushed into the column owners
  for (int base = 0; base < a.rowsA; base += NTEAM) {
    const int lb = base + team;
    const bool act = lb < nrows;
    float2* row = A1 + (act ? lb : 0) * RP;
    const int y = a.Blo + b0 + (act ? lb : 0);
    const int py = FftTeam<NL>::pidx(y);
    // crop x pupil straight into the registers of the transform's first pass (x = lane + TL j);
    // every load is issued before the first product
    constexpr int PL = FftTeam<NL>::P;
    float2 v[PL];
    if (act) {
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
    if (base == 0) {  // the twiddles (cp.async group 0) have landed and are visible CTA-wide
      if (has_meas) {
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
      __syncthreads();
    }
    team_fft_core<NL, true>(v, row, tw, lane, act);
    if (base == 0) cluster_wait<CS>();
    // the transform leaves X[k1 + P k2] in v[m Q + k2] (k1 = lane + Q m): a team's lanes hold
    // consecutive x, so each store below writes a contiguous run of the owner's row py
    if (act) {
      constexpr int Q = FftTeam<NL>::Q;
#pragma unroll
      for (int m = 0; m < PL / Q; ++m) {
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int x = lane + Q * m + PL * k2;
          const float2 val = v[m * Q + k2];
          const int own = x / CW, c = x - own * CW + 1;
          if constexpr (CS > 1) {
            const uint32_t e = smem_u32(OC + py * PO + c), m = smem_u32(&mbar[0]);
            st_async_f2(mapa_u32(e, own), val, mapa_u32(m, own));
            if (c == CW && own + 1 < CS)  // left halo of the next CTA
              st_async_f2(mapa_u32(e - 8u * CW, own + 1), val, mapa_u32(m, own + 1));
            if (c == 1 && own > 0)        // right halo of the previous CTA
              st_async_f2(mapa_u32(e + 8u * CW, own - 1), val, mapa_u32(m, own - 1));
          } else {
            OC[py * PO + c] = val;
          }
        }
      }
    }
  }
  if (a.rowsA <= 0) {  // no band rows (not produced by the host): still complete both waits
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    cluster_wait<CS>();
  }
  if constexpr (CS > 1) {
    mbar_wait_or_flag(&mbar[0], a.err);  // every band row of this CTA's columns has landed
  } else {
    __syncthreads();
  }

  // ---- B: inverse column transforms of the owned + halo columns (all local now);
  // only the support band rows hold data, the rest are zeros the transform never reads
  for (int base = 0; base < WC; base += NTEAM) {
    const int lc = base + team;
    const int x = x0 - 1 + lc;
    const bool act = (lc < WC) && x >= 0 && x < NL;
    team_fft<NL, true, PO>(OC + (act ? lc : 0), tw, lane, act, a.Blo, a.nb);
  }
  if (has_meas) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  // o = (-1)^(x+y) scale * IDFT.  The stencil only needs |o| and W = o w times the same
  // (-1)^(x+y) again (the forward shift), so the sign is never applied: o~ = scale * IDFT
  // gives |o~| = |o| and (-1)^(x+y) o w = o~ w.
  // The scale, 1 / (u^2 n^2), a power of two, was applied to stage A's input; a power of two commutes
  // exactly with every rounding of the transform, so this is bitwise scale * IDFT
  auto load_o = [&](int y, int c) -> float2 { return OC[FftTeam<NL>::pidx(y) * PO + c]; };
  if (a.mode == 1) {  // forward model only: |o|^2 on the owned columns
    for (int y = warp; y < NL; y += NW)
      for (int cc = wl; cc < CW; cc += 32) a.I_out[img + (size_t)y * NL + x0 + cc] = cabs2(load_o(y, cc + 1));
    return;  // no remote access after the last cluster barrier
  }
  // residual r = |o|^2 - I (Eq. 5), |o| - sqrt(max(I, 0)) (Eq. 4) or g(|o|^2) - g(max(I, 0)) (Sec. 6.3),
  // the measured side of Eq. 4 and of the maps mapped once per data set.  For the maps, sl = g'(|o|^2)
  // comes out of the same evaluation: the power map as p = max(|o|^2, eta^2)^(gamma - 1), g = |o|^2 p,
  // g' = gamma p (one powf per pixel); the log map as ln(1 + |o|^2) and 1 / (1 + |o|^2).
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

  // W = o * nabla^T omega (Eq. 11) or o / (2 max(|o|, eta)) * nabla^T omega (Eq. 10),
  // times (-1)^(x+y) for the forward shift; cost phi summed over owned pixels.
  // Each warp walks a strip of rows with its lanes on the owned columns, carrying
  // r, o and omega_y of the neighbouring rows in registers: the residual and the
  // normaliser are evaluated once per pixel, x-neighbours come by shuffle and the
  // halo columns are evaluated by the edge lanes.  The rows just outside the strip
  // are read before a block barrier, because their owners overwrite them with W.
  float acc = 0.f;  // per-thread partial of at most NL/SW pixels; block sum in FP64
  if (a.mode == 2) {
    // multiplexed images: W = o f, with f = g'(s_j) nabla^T omega of the LED's image computed once
    // per image beforehand (residual, normaliser and cost are per image, not per LED)
    for (int i = tid; i < NL * CW; i += NT) {
      const int y = i / CW, cc = i - y * CW;
      OC[FftTeam<NL>::pidx(y) * PO + cc + 1] = cscale(load_o(y, cc + 1), Itile[y * CW + cc]);
    }
  } else {
    static_assert(CW <= 32, "one warp spans the owned columns");
    constexpr int SW = pow2_floor(NW);  // strip warps; the others only take part in the barrier
    constexpr int RPW = NL / SW;        // rows per strip
    static_assert(RPW * SW == NL, "strips tile the rows");
    const float tau = a.tau, tau2 = fmaxf(a.tau * a.tau, 1e-36f), hit = (a.tau > 0.f) ? 0.5f / a.tau : 0.f;
    const bool on = wl < CW;
    const int cc = on ? wl : 0;
    const int c = cc + 1, x = x0 + cc;
    const bool has_left = x0 >= 1, has_right = x0 + CW < NL;
    const bool strip = warp < SW;
    const int ybeg = strip ? warp * RPW : 0, yend = strip ? ybeg + RPW : 0;  // empty strip: no rows
    auto r_own = [&](int y) { return resid(load_o(y, c), Itile[y * CW + cc]); };
    auto r_left = [&](int y) { return resid(load_o(y, 0), Ihalo[y]); };
    auto r_right = [&](int y) { return resid(load_o(y, CW + 1), Ihalo[NL + y]); };
    auto huber2 = [&](float dx, float dy) -> OmegaOut {
      OmegaOut o;
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
    // rows outside the strip, read before the barrier
    const float r_above = (strip && ybeg >= 1) ? r_own(ybeg - 1) : 0.f;
    const float r_below = (strip && yend < NL) ? r_own(yend) : 0.f;
    __syncthreads();
    if (strip) {
      float2 o_cur = load_o(ybeg, c);
      float sl_cur = 0.f, sl_nxt = 0.f;  // g'(|o|^2) of the current and next rows (Sec. 6.3 maps)
      float r_cur = resid_sl(o_cur, Itile[ybeg * CW + cc], sl_cur);
      // omega_y at the row above the strip (0 above the first row)
      float wy_prev = 0.f;
      if (ybeg >= 1) {
        float rr = __shfl_down_sync(0xffffffffu, r_above, 1);
        if (wl == CW - 1) rr = Hx[ybeg - 1];
        const float dx = (x < NL - 1) ? rr - r_above : 0.f;
        wy_prev = huber2(dx, r_cur - r_above).wy;
      }
      // the strip's rows, fully unrolled: only the last row's neighbour below depends on where
      // the strip lies (the next strip's first row, or the image edge, where dy = 0)
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
        const OmegaOut w0 = huber2(dx, dy);
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
  }  // mode 2 leaves acc = 0: the cost pairs of its LEDs are zero
  // the warps' cost pairs, summed in warp order by the last warp into one pair per CTA for the cost
  // reduction (below, after that warp's pushes)
  float2* cpair = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(Hx + 2 * NL) + 16);
  {
    const FF wsum = warp_sum_ff(FF{acc, 0.f});
    if (wl == 0) cpair[warp] = make_float2(wsum.hi, wsum.lo);
  }
  __syncthreads();  // W is complete in every column before the column transforms read it
  // forward column transforms of the owned columns (only the support band rows of the output are
  // written back: the other rows are never read), then push the band rows to their owners
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
      for (int m = 0; m < PL / Q; ++m) {
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int k = lane + Q * m + PL * k2;
          if ((unsigned)(k - a.Blo) < (unsigned)a.nb) col[FftTeam<NL>::pidx(k) * PO] = v[m * Q + k2];
        }
      }
    }
  }
  __syncthreads();
  for (int b = warp; b < a.nb; b += NW) {
    const int own = b / a.rowsA, lb = b - own * a.rowsA;
    const int py = FftTeam<NL>::pidx(a.Blo + b);
    for (int cc = wl; cc < CW; cc += 32) {
      float2* dst = A1 + lb * RP + FftTeam<NL>::pidx(x0 + cc);
      if constexpr (CS > 1) {
        st_async_f2(mapa_u32(smem_u32(dst), own), OC[py * PO + cc + 1], mapa_u32(smem_u32(&mbar[1]), own));
      } else {
        *dst = OC[py * PO + cc + 1];
      }
    }
  }
  // the CTA's cost pair: the warps' pairs summed in warp order by the last warp, after its pushes and
  // while the exchange completes
  if (tid == NT - 32) {
    FF s = {cpair[0].x, cpair[0].y};
    for (int w = 1; w < NW; ++w) s = ff_add(s, FF{cpair[w].x, cpair[w].y});
    a.cost_ff[(size_t)led * CS + crank] = make_float2(s.hi, s.lo);
  }
  if constexpr (CS > 1) {
    mbar_wait_or_flag(&mbar[1], a.err);  // all n columns of this CTA's band rows have landed
  } else {
    __syncthreads();
  }

  // ---- C: forward row transforms of this CTA's band rows; the support pixels go
  // from the transform's registers straight to G
  for (int base = 0; base < a.rowsA; base += NTEAM) {
    const int lb = base + team;
    const bool act = lb < nrows;
    float2* row = A1 + (act ? lb : 0) * RP;
    constexpr int PL = FftTeam<NL>::P, Q = FftTeam<NL>::Q;
    float2 v[PL];
    if (act) {
#pragma unroll
      for (int j = 0; j < PL; ++j) v[j] = row[lane + (Q + 1) * j];
    }
    team_fft_core<NL, false>(v, row, tw, lane, act);
    if (act) {
      const int ky = a.Blo + b0 + lb;
      const int xs = a.row_xs[ky], cnt = a.row_cnt[ky];
      float2* dst = a.G + (size_t)led * a.S + a.row_off[ky];
#pragma unroll
      for (int m = 0; m < PL / Q; ++m) {
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int d = lane + Q * m + PL * k2 - xs;
          if ((unsigned)d < (unsigned)cnt) dst[d] = cscale(v[m * Q + k2], a.scale);
        }
      }
    }
  }
}

int tile_cluster_size(int n) {
  switch (n) {
    case 256: return TileCfg<256>::CS;
    case 128: return TileCfg<128>::CS;
    case 64: return TileCfg<64>::CS;
    default: return 1;
  }
}

static int tile_threads(int n) {
  switch (n) {
    case 256: return TileCfg<256>::NT;
    case 128: return TileCfg<128>::NT;
    case 64: return TileCfg<64>::NT;
    default: return 256;
  }
}

size_t tile_smem_bytes(int n, int cs, int rowsA) {
  const size_t rp = fft_padded_length(n);
  const size_t cw = n / cs;
  return 4 * (size_t)n * (cw + 2) + 8 * ((size_t)n + (size_t)rowsA * rp + rp * (size_t)oc_pitch(n)) +
         4 * 2 * (size_t)n + 16 + 8 * (size_t)tile_warps(n);  // ... + Hx + two mbarriers + cost pairs
}

int tile_warps(int n) { return tile_threads(n) / 32; }

template <int NL>
static cudaError_t launch_tile_t(const TileArgs& a, cudaStream_t s) {
  constexpr int CS = TileCfg<NL>::CS, NT = TileCfg<NL>::NT;
  const size_t smem = tile_smem_bytes(NL, CS, a.rowsA);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.nled > 0 ? a.nled : a.K) * CS);
  cfg.blockDim = dim3(NT);
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
  const int fid = (a.fidelity >= 2) ? 2 : a.fidelity;
  const int var = (a.mode != 0) ? 1 : 2 * fid + (a.iso ? 1 : 0);  // modes 1, 2 skip the stencil
  switch (var) {
    case 0: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 0, 0>, a);
    case 1: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 0, 1>, a);
    case 2: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 1, 0>, a);
    case 3: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 1, 1>, a);
    case 4: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 2, 0>, a);
    default: return cudaLaunchKernelEx(&cfg, tile_kernel<NL, CS, NT, 2, 1>, a);
  }
}

template <int NL>
static cudaError_t prepare_tile_t(int rowsA) {
  constexpr int CS = TileCfg<NL>::CS, NT = TileCfg<NL>::NT;
  static int configured = 0;  // largest dynamic shared memory size set so far
  const int smem = (int)tile_smem_bytes(NL, CS, rowsA);
  if (smem <= configured) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (auto k : {tile_kernel<NL, CS, NT, 0, 0>, tile_kernel<NL, CS, NT, 0, 1>, tile_kernel<NL, CS, NT, 1, 0>,
                 tile_kernel<NL, CS, NT, 1, 1>, tile_kernel<NL, CS, NT, 2, 0>, tile_kernel<NL, CS, NT, 2, 1>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) configured = smem;
  return e;
}

cudaError_t prepare_tile(int n, int rowsA) {
  switch (n) {
    case 16: return prepare_tile_t<16>(rowsA);
    case 32: return prepare_tile_t<32>(rowsA);
    case 64: return prepare_tile_t<64>(rowsA);
    case 128: return prepare_tile_t<128>(rowsA);
    case 256: return prepare_tile_t<256>(rowsA);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile(const TileArgs& a, int n, cudaStream_t s) {
  switch (n) {
    case 16: return launch_tile_t<16>(a, s);
    case 32: return launch_tile_t<32>(a, s);
    case 64: return launch_tile_t<64>(a, s);
    case 128: return launch_tile_t<128>(a, s);
    case 256: return launch_tile_t<256>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace elf
