// Spectrum-sized kernels of one Elfpie iteration and its set-up:
//   hessian_kernel   Eqs. 6-7 costs and the object-domain factors of Eqs. 13-14 (tiles in shared
//                    memory; hessian_walk_kernel: the same per column in registers, from N = 512)
//   gather_kernel    Eq. 9's sum over LEDs (fixed ascending order, no atomics)
//                    fused with the Eq. 19 update of Psi (g = Eq. 15)
//   pupil kernels    Eq. 18 in fixed LED chunks, the 3x3 Gaussian smoothing of P
//                    (note under Algorithm 1) and Eq. 19 for P
//   cost_reduce      Eq. 8's three terms in FP64, fixed order
//   alpha kernels    Eqs. 16-17 in FP64, fixed order
//   init kernels     the initial state of elf_set_measurements
#include <algorithm>

#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace elf {

// ------------------------------------------------------------------ helpers
// Fixed-order block sum (1D or 2D blocks of whole warps, at most 8 warps);
// the result is valid in the block's first thread.
__device__ __forceinline__ double block_sum_double(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int w = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
  __syncthreads();
  if ((t & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (t == 0)
    for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Smoothed L1 of a 3-vector (reading A7): cost and omega = h / max(|h|, tau)
// (isotropic), or the same rule per component (anisotropic).  hit = 1 / (2 tau) (0 when tau = 0,
// where the quadratic branch is never taken), hoisted out of the per-pixel work.
__device__ __forceinline__ float huber3(float& h0, float& h1, float& h2, float tau, float hit, int iso) {
  if (iso) {
    const float ss = h0 * h0 + h1 * h1 + h2 * h2;
    const float inv = rsqrtf(fmaxf(ss, fmaxf(tau * tau, 1e-36f)));
    h0 *= inv;
    h1 *= inv;
    h2 *= inv;
    return (ss >= tau * tau) ? ss * inv : ss * hit + 0.5f * tau;
  }
  float c = 0.f;
  float* hs[3] = {&h0, &h1, &h2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float a = fabsf(*hs[i]);
    c += (a >= tau) ? a : a * a * hit + 0.5f * tau;
    *hs[i] /= fmaxf(a, fmaxf(tau, 1e-18f));  // 0 at the origin when tau = 0
  }
  return c;
}

// ------------------------------------------------------------------ Hessian (Eqs. 6-7, 13-14)
constexpr int HT = 16;            // output tile side (16 x 16 blocks: 64/256/49 at 24.7 against 27.0 us per
                                  // iteration with 32 x 32 tiles and 32 x 8 blocks)
constexpr int HA = HT + 4;        // amplitude/phase tile with a 2-pixel halo
constexpr int HW = HT + 2;        // omega tile with a 1-pixel halo

// Block of HT x (256 / HT) threads per HT x HT output tile (2-pixel halo).
__global__ void __launch_bounds__(256) hessian_kernel(const HessArgs a) {
  __shared__ float s_a[HA][HA + 1];
  __shared__ float s_p[HA][HA + 1];
  __shared__ float s_w[6][HW][HW + 1];
  __shared__ float red[4 * 8];
  const int N = a.N;
  const int tx0 = blockIdx.x * HT, ty0 = blockIdx.y * HT;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * HT + tx;
  const float alpha = (float)a.weights[0], beta = (float)a.weights[1];
  const float hit = a.tau > 0.f ? 0.5f / a.tau : 0.f;
  pdl_launch_dependents();
  pdl_wait();  // the column pass wrote ot

  // O = (-1)^(x+y) Ot / A; amplitude and phase (atan2, reading A12)
  for (int i = tid; i < HA * HA; i += 256) {
    {
      const int ly = i / HA, lx = i - ly * HA;
      const int y = ty0 - 2 + ly, x = tx0 - 2 + lx;
      float am = 0.f, ph = 0.f;
      if (y >= 0 && y < N && x >= 0 && x < N) {
        float2 o = a.ot[(size_t)y * N + x];
        const float sg = ((x + y) & 1) ? -a.invA : a.invA;
        o.x *= sg;
        o.y *= sg;
        am = sqrtf(cabs2(o));
        ph = atan2f(o.y, o.x);
      }
      s_a[ly][lx] = am;
      s_p[ly][lx] = ph;
    }
  }
  __syncthreads();

  // omega = H f / max(|H f|, tau) on the interior [1, N-2]^2, zero elsewhere;
  // per-thread cost partials in FP32 (a handful of pixels), block sums in FP64
  float ca = 0.f, cp = 0.f;
  const float r2 = 1.41421356237309505f;
  for (int i = tid; i < HW * HW; i += 256) {
    {
      const int ly = i / HW, lx = i - ly * HW;
      const int y = ty0 - 1 + ly, x = tx0 - 1 + lx;
      const int cy = ly + 1, cx = lx + 1;  // centre in the HA tile
      float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (y >= 1 && y <= N - 2 && x >= 1 && x <= N - 2) {
        float h0 = s_a[cy][cx - 1] - 2.f * s_a[cy][cx] + s_a[cy][cx + 1];
        float h1 = s_a[cy - 1][cx] - 2.f * s_a[cy][cx] + s_a[cy + 1][cx];
        float h2 = r2 * 0.25f * (s_a[cy + 1][cx + 1] - s_a[cy + 1][cx - 1] - s_a[cy - 1][cx + 1] + s_a[cy - 1][cx - 1]);
        const float fa = huber3(h0, h1, h2, a.tau, hit, a.iso);
        float g0 = s_p[cy][cx - 1] - 2.f * s_p[cy][cx] + s_p[cy][cx + 1];
        float g1 = s_p[cy - 1][cx] - 2.f * s_p[cy][cx] + s_p[cy + 1][cx];
        float g2 = r2 * 0.25f * (s_p[cy + 1][cx + 1] - s_p[cy + 1][cx - 1] - s_p[cy - 1][cx + 1] + s_p[cy - 1][cx - 1]);
        const float fp = huber3(g0, g1, g2, a.tau, hit, a.iso);
        w[0] = h0; w[1] = h1; w[2] = h2; w[3] = g0; w[4] = g1; w[5] = g2;
        if (ly >= 1 && ly <= HT && lx >= 1 && lx <= HT) {  // owned pixel
          ca += fa;
          cp += fp;
        }
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) s_w[k][ly][lx] = w[k];
    }
  }
  __syncthreads();

  // q = alpha O/(2 max(a,eta)) H^T omega_a + beta (i/2) O/(a^2+eta) H^T omega_phi
  for (int ly = ty; ly < HT; ly += 256 / HT) {
    const int lx = tx;
    const int y = ty0 + ly, x = tx0 + lx;
    if (y >= N || x >= N) continue;
    const int wy = ly + 1, wx = lx + 1;
    float t[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const int k = 3 * f;
      const float dxx = s_w[k][wy][wx - 1] - 2.f * s_w[k][wy][wx] + s_w[k][wy][wx + 1];
      const float dyy = s_w[k + 1][wy - 1][wx] - 2.f * s_w[k + 1][wy][wx] + s_w[k + 1][wy + 1][wx];
      const float dxy = s_w[k + 2][wy - 1][wx - 1] - s_w[k + 2][wy - 1][wx + 1] - s_w[k + 2][wy + 1][wx - 1] +
                        s_w[k + 2][wy + 1][wx + 1];
      t[f] = dxx + dyy + r2 * 0.25f * dxy;
    }
    const float am = s_a[ly + 2][lx + 2];
    float2 o = a.ot[(size_t)y * N + x];
    const float sg = ((x + y) & 1) ? -a.invA : a.invA;
    o.x *= sg;
    o.y *= sg;
    const float ka = __fdividef(alpha * t[0], 2.f * fmaxf(am, a.eta));
    const float kp = __fdividef(beta * 0.5f * t[1], am * am + a.eta);
    // ka O + i kp O, then the forward-shift sign and 1/A
    float2 q = make_float2(ka * o.x - kp * o.y, ka * o.y + kp * o.x);
    a.q[(size_t)y * N + x] = cscale(q, sg);
  }
  (void)tid;
  const float part[2] = {ca, cp};
  double sum[2];
  block_sum_ff<2>(part, red, sum);
  if (tid == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    a.costpart[2 * b] = sum[0];
    a.costpart[2 * b + 1] = sum[1];
  }
}

// The same computation without shared memory, so that its blocks fit beside the tile kernels' on one SM.
// Each thread owns one column and walks a strip of ROWS output rows, keeping in registers a 3-row
// window of a = |O| and phi = atan2(O) (with the left and right neighbours' values, exchanged by warp
// shuffles), a 3-row window of omega, and the rows of O it still needs.  A warp spans 32 columns; its
// 28 inner lanes are outputs and the two outer lanes per side supply the neighbours' a, phi and
// omega.  Every a and phi is computed once per warp, every omega once, and each pixel's cost is
// counted by the one lane and row that own it.
constexpr int kWalkOut = 28;    // output columns per warp
constexpr int kWalkWarps = 2;   // warps per block: 64 threads fit beside two column CTAs of the tile work

struct WalkAP {  // a and phi of one row at the thread's column and its two neighbours
  float aL, aM, aR, pL, pM, pR;
};
struct WalkW {   // omega of one row (one field): the components Hᵀ needs, with neighbours
  float xxL, xxM, xxR, yy, xyL, xyR;
};

__device__ __forceinline__ void walk_ap(const HessArgs& a, int x, int r, WalkAP& o, float2& Or) {
  const int N = a.N;
  float am = 0.f, ph = 0.f;
  Or = make_float2(0.f, 0.f);
  if (r >= 0 && r < N && x >= 0 && x < N) {
    float2 v = a.ot[(size_t)r * N + x];
    const float sg = ((x + r) & 1) ? -a.invA : a.invA;
    v.x *= sg;
    v.y *= sg;
    Or = v;
    am = sqrtf(cabs2(v));
    ph = atan2f(v.y, v.x);
  }
  o.aM = am;
  o.pM = ph;
  o.aL = __shfl_up_sync(0xffffffffu, am, 1);
  o.aR = __shfl_down_sync(0xffffffffu, am, 1);
  o.pL = __shfl_up_sync(0xffffffffu, ph, 1);
  o.pR = __shfl_down_sync(0xffffffffu, ph, 1);
}

// omega of row r (rows r - 1, r, r + 1 of a and phi given) for both fields; the smoothed cost of the
// pixel is added when count is set.  Zero outside the interior.
__device__ __forceinline__ void walk_omega(const HessArgs& a, float hit, bool inside, bool count, const WalkAP& u,
                                           const WalkAP& m, const WalkAP& d, WalkW& wa, WalkW& wp, float& ca,
                                           float& cp) {
  const float r2 = 1.41421356237309505f;
  float h0 = 0.f, h1 = 0.f, h2 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (inside) {
    h0 = m.aL - 2.f * m.aM + m.aR;
    h1 = u.aM - 2.f * m.aM + d.aM;
    h2 = r2 * 0.25f * (d.aR - d.aL - u.aR + u.aL);
    const float fa = huber3(h0, h1, h2, a.tau, hit, a.iso);
    g0 = m.pL - 2.f * m.pM + m.pR;
    g1 = u.pM - 2.f * m.pM + d.pM;
    g2 = r2 * 0.25f * (d.pR - d.pL - u.pR + u.pL);
    const float fp = huber3(g0, g1, g2, a.tau, hit, a.iso);
    if (count) {
      ca += fa;
      cp += fp;
    }
  }
  wa.xxM = h0;
  wa.yy = h1;
  wp.xxM = g0;
  wp.yy = g1;
  wa.xxL = __shfl_up_sync(0xffffffffu, h0, 1);
  wa.xxR = __shfl_down_sync(0xffffffffu, h0, 1);
  wa.xyL = __shfl_up_sync(0xffffffffu, h2, 1);
  wa.xyR = __shfl_down_sync(0xffffffffu, h2, 1);
  wp.xxL = __shfl_up_sync(0xffffffffu, g0, 1);
  wp.xxR = __shfl_down_sync(0xffffffffu, g0, 1);
  wp.xyL = __shfl_up_sync(0xffffffffu, g2, 1);
  wp.xyR = __shfl_down_sync(0xffffffffu, g2, 1);
}

// H^T omega at the middle row of three omega rows.
__device__ __forceinline__ float walk_ht(const WalkW& u, const WalkW& m, const WalkW& d) {
  const float dxx = m.xxL - 2.f * m.xxM + m.xxR;
  const float dyy = u.yy - 2.f * m.yy + d.yy;
  const float dxy = u.xyL - u.xyR - d.xyL + d.xyR;
  return dxx + dyy + 1.41421356237309505f * 0.25f * dxy;
}

template <int ROWS>
__global__ void __launch_bounds__(32 * kWalkWarps) hessian_walk_kernel(const HessArgs a) {
  __shared__ float red[2 * 2 * kWalkWarps];
  const int N = a.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = (blockIdx.x * kWalkWarps + warp) * kWalkOut - 2 + lane;
  const int y0 = blockIdx.y * ROWS;
  const bool xint = x >= 1 && x <= N - 2;
  const bool own = lane >= 2 && lane < 2 + kWalkOut && x < N;
  const float alpha = (float)a.weights[0], beta = (float)a.weights[1];
  float ca = 0.f, cp = 0.f;
  const float hit = a.tau > 0.f ? 0.5f / a.tau : 0.f;
  pdl_launch_dependents();
  pdl_wait();  // the column pass wrote ot
  // windows: a / phi of rows y, y + 1, y + 2 (A0, A1, A2), omega of rows y - 1, y, y + 1 (W*0, W*1, W*2),
  // O of rows y, y + 1, y + 2
  WalkAP A0, A1, A2, Am;
  float2 O0, O1, O2, Od;
  walk_ap(a, x, y0 - 2, Am, Od);
  walk_ap(a, x, y0 - 1, A0, Od);
  walk_ap(a, x, y0, A1, O1);
  walk_ap(a, x, y0 + 1, A2, O2);
  WalkW Wa0, Wa1, Wa2, Wp0, Wp1, Wp2;
  {
    const int r = y0 - 1;
    walk_omega(a, hit, xint && r >= 1 && r <= N - 2, false, Am, A0, A1, Wa1, Wp1, ca, cp);
    const int r1 = y0;
    walk_omega(a, hit, xint && r1 >= 1 && r1 <= N - 2, own && r1 < N, A0, A1, A2, Wa2, Wp2, ca, cp);
  }
  // shift: a / phi rows y0 .. y0 + 1 into A0 .. A1, O likewise
  A0 = A1;
  A1 = A2;
  O0 = O1;
  O1 = O2;
#pragma unroll 4
  for (int i = 0; i < ROWS; ++i) {
    const int y = y0 + i;
    // a / phi and O of row y + 2
    walk_ap(a, x, y + 2, A2, O2);
    // omega of row y + 1 (counted when that row is an output row of this strip)
    Wa0 = Wa1;
    Wp0 = Wp1;
    Wa1 = Wa2;
    Wp1 = Wp2;
    const int r = y + 1;
    walk_omega(a, hit, xint && r >= 1 && r <= N - 2, own && i + 1 < ROWS && r < N, A0, A1, A2, Wa2, Wp2, ca, cp);
    // q of row y: alpha O / (2 max(a, eta)) H^T omega_a + beta (i/2) O / (a^2 + eta) H^T omega_phi,
    // times (-1)^(x+y) / A for the forward transform
    if (own && y < N) {
      const float ta = walk_ht(Wa0, Wa1, Wa2), tp = walk_ht(Wp0, Wp1, Wp2);
      const float am = A0.aM;
      const float2 o = O0;
      const float sg = ((x + y) & 1) ? -a.invA : a.invA;
      const float ka = __fdividef(alpha * ta, 2.f * fmaxf(am, a.eta));
      const float kp = __fdividef(beta * 0.5f * tp, am * am + a.eta);
      const float2 q = make_float2(ka * o.x - kp * o.y, ka * o.y + kp * o.x);
      a.q[(size_t)y * N + x] = cscale(q, sg);
    }
    A0 = A1;
    A1 = A2;
    O0 = O1;
    O1 = O2;
  }
  const float part[2] = {ca, cp};
  double sum[2];
  block_sum_ff<2>(part, red, sum);
  if (threadIdx.x == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    a.costpart[2 * b] = sum[0];
    a.costpart[2 * b + 1] = sum[1];
  }
}

static int walk_cols(int N) { return (((N + kWalkOut - 1) / kWalkOut) + kWalkWarps - 1) / kWalkWarps; }

// Which kernel runs, measured on GB300 in the whole iteration: the tiled kernel at N <= 256 (64/256/49:
// 29.5 against 30.8 us), the walk with 8-row strips at N = 512 (52.7 against 53.4 us at 128/512/225)
// and with 16-row strips from N = 1024 (161.0 against 163.0 us at 256/1024/225; 32-row strips shorten
// the tile stage but end the branch later: 0.168 against 0.164 ms per step).  Shorter strips give more
// warps for latency hiding and cost recomputed halo rows.
static int walk_rows(int N) { return N <= 256 ? 0 : (N <= 512 ? 8 : 16); }

// Blocks of the launch, each writing one (L_A, L_Phi) cost pair.
int hess_blocks(int N) {
  const int r = walk_rows(N);
  if (r == 0) return ((N + HT - 1) / HT) * ((N + HT - 1) / HT);
  return walk_cols(N) * ((N + r - 1) / r);
}

cudaError_t launch_hessian(const HessArgs& a, cudaStream_t s, bool pdl) {
  const int r = walk_rows(a.N);
  if (r == 0) {
    const int t = (a.N + HT - 1) / HT;
    if (pdl) return launch_dependent(hessian_kernel, dim3(t, t), dim3(HT, 256 / HT), 0, s, a);
    hessian_kernel<<<dim3(t, t), dim3(HT, 256 / HT), 0, s>>>(a);
  } else if (r == 8) {
    if (pdl) return launch_dependent(hessian_walk_kernel<8>, dim3(walk_cols(a.N), (a.N + 7) / 8), dim3(32 * kWalkWarps), 0, s, a);
    hessian_walk_kernel<8><<<dim3(walk_cols(a.N), (a.N + 7) / 8), 32 * kWalkWarps, 0, s>>>(a);
  } else {
    if (pdl) return launch_dependent(hessian_walk_kernel<16>, dim3(walk_cols(a.N), (a.N + 15) / 16), dim3(32 * kWalkWarps), 0, s, a);
    hessian_walk_kernel<16><<<dim3(walk_cols(a.N), (a.N + 15) / 16), 32 * kWalkWarps, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gather + AdaBelief (Eqs. 9, 15, 19)
// Eq. 19 for one complex parameter; returns the increment Delta.
__device__ __forceinline__ float2 adabelief_step(float2 g, float2& mu, float& v, float& delta, float g1, float g2,
                                                 float eta, float bc1, float bc2) {
  mu = make_float2(g1 * mu.x + (1.f - g1) * g.x, g1 * mu.y + (1.f - g1) * g.y);
  const float ex = mu.x - g.x, ey = mu.y - g.y;
  v = g2 * v + (1.f - g2) * (ex * ex + ey * ey);
  const float vhat = v * bc2;
  const float k = (sqrtf(delta) + eta) / (sqrtf(vhat) + eta);
  const float2 d = make_float2(k * (g1 * mu.x * bc1 + (1.f - g1) * g.x), k * (g1 * mu.y * bc1 + (1.f - g1) * g.y));
  delta = g1 * delta + (1.f - g1) * cabs2(d);
  return d;
}

// Two horizontally adjacent spectrum pixels per thread (16-byte state loads and stores); the
// threads of a row segment (64 pixels: one warp) walk that segment's list, which holds exactly the
// LEDs whose support chord crosses it, in ascending order.
// Block rows run from the centre of the spectrum outwards: the central rows are crossed by the most
// LEDs and take longest, so they are dispatched first and the short outer rows fill the tail.
__global__ void __launch_bounds__(256, 5) gather_kernel(const GatherArgs a) {
  const int seg_w = 2 * blockDim.x;
  const int x = blockIdx.x * seg_w + 2 * threadIdx.x;  // first of the thread's two pixels
  const int by = blockIdx.y, cb = gridDim.y >> 1;
  const int rb = (by & 1) ? cb - ((by + 1) >> 1) : cb + (by >> 1);  // covers [0, gridDim.y) for even counts
  const int y = rb * blockDim.y + threadIdx.y;
  const size_t k = (size_t)y * a.N + x;
  // the Eq. 19 state is read after the LED loop; ask L2 for it now so the loop covers its latency
  if (a.mode == 0) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.mu + k));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.v + k));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.delta + k));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psi + k));
  }
  const int seg = y * a.tiles_x + blockIdx.x;
  const int e0 = a.seg_ptr[seg], e1 = a.seg_ptr[seg + 1];
  // covering LEDs in ascending order; the loads of two entries are issued before their products
  // are added (same additions in the same order as one entry at a time).  Few loads in flight per
  // thread and 47 registers: five blocks per SM, whose warps hide the latency
  float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
  constexpr int U = 2;
  // the segment's entries, 32 at a time, one per lane, handed round by shuffles: only the G and
  // pupil loads of a round wait on memory (a warp is one row segment when the segment has 64 pixels;
  // with 32-pixel segments two rows share a warp and each half-warp shuffles within itself)
  const int lanes = min((int)blockDim.x, 32);
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int lane_base = lane & ~(lanes - 1);
  const unsigned wmask = (lanes == 32) ? 0xffffffffu : (0xffffu << lane_base);
  for (int c0 = e0; c0 < e1; c0 += lanes) {
    const int cl = lane - lane_base;
    const int4 mine = (c0 + cl < e1) ? __ldg(&a.seg_ent[c0 + cl]) : make_int4(0, 0, 0, 0);
    const int c1 = min(e1, c0 + lanes);
  for (int i0 = c0; i0 < c1; i0 += U) {
    float2 p0[U], g0[U], p1[U], g1[U];
    bool ok0[U], ok1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ok0[u] = ok1[u] = false;
      p0[u] = g0[u] = p1[u] = g1[u] = make_float2(0.f, 0.f);
      const int src = lane_base + min(i0 + u - c0, lanes - 1);
      int4 e;
      e.x = __shfl_sync(wmask, mine.x, src);
      e.y = __shfl_sync(wmask, mine.y, src);
      e.z = __shfl_sync(wmask, mine.z, src);
      e.w = __shfl_sync(wmask, mine.w, src);
      if (i0 + u < c1) {
        const int lo = e.w & 0xffff, cnt = e.w >> 16;
        const float2* gp = a.G + (size_t)e.x * a.S + e.y;
        if ((unsigned)(x - lo) < (unsigned)cnt) {
          ok0[u] = true;
          p0[u] = a.pupil[e.z + x];
          g0[u] = gp[x];
        }
        if ((unsigned)(x + 1 - lo) < (unsigned)cnt) {
          ok1[u] = true;
          p1[u] = a.pupil[e.z + x + 1];
          g1[u] = gp[x + 1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ok0[u]) acc0 = cadd(acc0, cconjmul(p0[u], g0[u]));
      if (ok1[u]) acc1 = cadd(acc1, cconjmul(p1[u], g1[u]));
    }
  }
  }
  // the state after the LED loop, so that the loop's loads and the state do not hold registers at the
  // same time (occupancy hides the latency instead)
  const float4 g = a.gH ? *reinterpret_cast<const float4*>(a.gH + k) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 mu = make_float4(0.f, 0.f, 0.f, 0.f), ps = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 v = make_float2(0.f, 0.f), dl = make_float2(0.f, 0.f);
  if (a.mode == 0) {
    mu = *reinterpret_cast<const float4*>(a.mu + k);
    v = *reinterpret_cast<const float2*>(a.v + k);
    dl = *reinterpret_cast<const float2*>(a.delta + k);
    ps = *reinterpret_cast<const float4*>(a.psi + k);
  }
  float2 ga = cadd(make_float2(g.x, g.y), acc0), gb = cadd(make_float2(g.z, g.w), acc1);
  if (a.mode == 1) {
    *reinterpret_cast<float4*>(a.g_out + k) = make_float4(ga.x, ga.y, gb.x, gb.y);
    return;
  }
  float2 mua = make_float2(mu.x, mu.y), mub = make_float2(mu.z, mu.w);
  const float2 da = adabelief_step(ga, mua, v.x, dl.x, a.g1, a.g2, a.eta, a.bc[0], a.bc[1]);
  const float2 db = adabelief_step(gb, mub, v.y, dl.y, a.g1, a.g2, a.eta, a.bc[0], a.bc[1]);
  const float part[2] = {cabs2(ga) + cabs2(gb), cabs2(da) + cabs2(db)};
  *reinterpret_cast<float4*>(a.psi_out + k) = make_float4(ps.x - da.x, ps.y - da.y, ps.z - db.x, ps.w - db.y);
  *reinterpret_cast<float4*>(a.mu + k) = make_float4(mua.x, mua.y, mub.x, mub.y);
  *reinterpret_cast<float2*>(a.v + k) = v;
  *reinterpret_cast<float2*>(a.delta + k) = dl;

  // ||g|| and ||Delta Psi|| of this iteration: each block's FP32 sums of |g|^2 and |Delta|^2 (a fixed
  // tree over its 512 positive terms: relative error at most 9 * 2^-24), added in block order with
  // error-free pair sums by the next cost reduction (norms_finalize)
  __shared__ float2 red[8];
  float s0 = part[0], s1 = part[1];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, off);
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) red[tid >> 5] = make_float2(s0, s1);
  __syncthreads();
  if (tid == 0) {
    float2 t = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) t = make_float2(t.x + red[w].x, t.y + red[w].y);
    a.norm_part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    if (blockIdx.x == 0 && blockIdx.y == 0) *a.norm_pending = 1;
  }
}

// The norms of an update from its gather's block partials: the blocks in index order (eight loads
// in flight per thread, then one block sum), square roots into the next ring slot.  One block; every
// thread calls it.  A no-op when no partials are pending.
__device__ void norms_finalize(const float2* part, int nblk, int* pending, int* slot, double* ring, float* red) {
  if (*pending == 0) return;  // the same value for every thread: no kernel beside this one writes it
  const int tid = threadIdx.x, nt = blockDim.x;
  FF t[2] = {{0.f, 0.f}, {0.f, 0.f}};
  constexpr int U = 8;
  for (int i0 = tid; i0 < nblk; i0 += U * nt) {
    float2 p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) p[u] = (i0 + u * nt < nblk) ? __ldcg(part + i0 + u * nt) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + u * nt < nblk) {
        t[0] = ff_add(t[0], FF{p[u].x, 0.f});
        t[1] = ff_add(t[1], FF{p[u].y, 0.f});
      }
    }
  }
  double nrm[2];
  block_sum_ff<2>(t, red, nrm);
  if (tid == 0) {
    const int it = *slot;
    ring[2 * (it % kCostRing)] = sqrt(nrm[0]);
    ring[2 * (it % kCostRing) + 1] = sqrt(nrm[1]);
    *slot = it + 1;
    *pending = 0;
  }
}

__global__ void __launch_bounds__(256) norms_finalize_kernel(const float2* part, int nblk, int* pending, int* slot,
                                                              double* ring) {
  __shared__ float red[2 * 2 * 8];
  norms_finalize(part, nblk, pending, slot, ring, red);
}

cudaError_t launch_norms_finalize(const NormArgs& n, cudaStream_t s) {
  norms_finalize_kernel<<<1, 256, 0, s>>>(n.part, n.nblk, n.pending, n.slot, n.ring);
  return cudaGetLastError();
}

int gather_blocks(int N) { return N * N / 512; }  // 512 pixels per block (see launch_gather)

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s) {
  const int seg = gather_seg(a.N);          // 64, or 32 for a 32 x 32 spectrum
  const dim3 block(seg / 2, 256 / (seg / 2)); // one thread per two pixels of a segment
  const dim3 grid(a.tiles_x, a.N / block.y);  // gather_blocks(N) blocks in all
  gather_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ pupil (Eq. 18, Eq. 19, Gaussian filter)
int pupil_chunks(int K, int S) {
  // enough (support pixel, LED chunk) pairs to fill the GPU, chunks of >= 4 LEDs
  int q = (4 * 152 * 256 + S - 1) / (S > 0 ? S : 1);
  if (q > K / 4) q = K / 4;
  if (q < 1) q = 1;
  return q;
}

// Eq. 19 for one pupil pixel j with gradient g (zero off the support): the 3x3 Gaussian of P^t
// (note under Algorithm 1) as the base, P^(t+1) = mask o (base - Delta); gradient mode writes g.
__device__ __forceinline__ void pupil_update_pixel(const PupilArgs& a, int j, float2 g, bool on_support) {
  if (a.mode == 1) {
    a.g_out[j] = g;
    return;
  }
  const int n = a.n;
  const int jy = j / n, jx = j - jy * n;
  float2 base;
  if (a.filter) {
    base = make_float2(0.f, 0.f);
    const float w[3] = {a.w1, a.w0, a.w1};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int yy = jy + dy, xx = jx + dx;
        if (yy < 0 || yy >= n || xx < 0 || xx >= n) continue;
        base = cadd(base, cscale(a.pupil[yy * n + xx], w[dy + 1] * w[dx + 1]));
      }
    }
  } else {
    base = a.pupil[j];
  }
  float2 mu = a.mu[j];
  float v = a.v[j], dl = a.delta[j];
  const float2 d = adabelief_step(g, mu, v, dl, a.g1, a.g2, a.eta, a.bc[0], a.bc[1]);
  a.mu[j] = mu;
  a.v[j] = v;
  a.delta[j] = dl;
  a.pupil_next[j] = on_support ? csub(base, d) : make_float2(0.f, 0.f);
}

// Eq. 18 in LED chunks: block (x, q) sums chunk q's LEDs for 256 support pixels.  The last block of
// each column of blocks to finish (a counter per column, reset by that block) then sums the Q
// partials of its pixels in chunk order and applies Eq. 19: no second launch, and the same sums in
// the same order whichever block is last.
__global__ void __launch_bounds__(256) pupil_partial_kernel(const PupilArgs a) {
  __shared__ int last;
  const int s = blockIdx.x * 256 + threadIdx.x;
  const bool valid = s < a.S;
  const int q = blockIdx.y;
  const int kc = (a.K + a.Q - 1) / a.Q;
  const int k0 = q * kc, k1 = min(a.K, k0 + kc);
  const int jy = valid ? a.sup_y[s] : 0, jx = valid ? a.sup_x[s] : 0;
  // LEDs in ascending order; four at a time have their loads in flight together
  float2 acc = make_float2(0.f, 0.f);
  constexpr int U = 4;
  for (int k = k0; valid && k < k1; k += U) {
    float2 ps[U], gt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ps[u] = gt[u] = make_float2(0.f, 0.f);
      if (k + u < k1) {
        const int2 o = a.origin[k + u];
        ps[u] = a.psi[(size_t)(o.x + jy) * a.N + o.y + jx];
        gt[u] = a.G[(size_t)(k + u) * a.S + s];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k + u < k1) acc = cadd(acc, cconjmul(ps[u], gt[u]));
  }
  if (valid) a.part[(size_t)q * a.S + s] = acc;
  __threadfence();  // the partial is visible device-wide before this block is counted
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&a.done[blockIdx.x], 1) == a.Q - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (valid) {
    float2 g = make_float2(0.f, 0.f);
    constexpr int V = 8;  // loads of eight chunks in flight, added in chunk order
    for (int q0 = 0; q0 < a.Q; q0 += V) {
      float2 pv[V];
#pragma unroll
      for (int u = 0; u < V; ++u)
        pv[u] = (q0 + u < a.Q) ? __ldcg(&a.part[(size_t)(q0 + u) * a.S + s]) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (q0 + u < a.Q) g = cadd(g, pv[u]);
    }
    pupil_update_pixel(a, jy * a.n + jx, g, true);
  }
  if (threadIdx.x == 0) a.done[blockIdx.x] = 0;  // ready for the next launch
}

// Eq. 19 for the pixels off the support (gradient 0; P^(t+1) = 0 there): needs nothing from the
// tile kernel, so it runs at the start of the pupil chain.
__global__ void __launch_bounds__(256) pupil_offsupport_kernel(const PupilArgs a) {
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= a.n * a.n || a.sidx_map[j] >= 0) return;
  pupil_update_pixel(a, j, make_float2(0.f, 0.f), false);
}

cudaError_t launch_pupil_partial(const PupilArgs& a, cudaStream_t s) {
  dim3 grid((a.S + 255) / 256, a.Q);
  pupil_partial_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pupil_offsupport(const PupilArgs& a, cudaStream_t s) {
  pupil_offsupport_kernel<<<(a.n * a.n + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Eq. 8 costs in FP64
// Sums the partials of Eq. 8's three terms in a fixed order into the cost ring (at
// iteration t) and/or out3.  It runs beside the gather and pupil kernels, on the stream of
// the Hessian branch.  With bc_next it also closes the iteration: t += 1, the running powers
// gp = (gamma1^(t+1), gamma2^(t+1)) and the next iteration's Eq. 19 bias corrections, written to the
// other half of the double-buffered pair (the gather and pupil kernels still read this one).
__global__ void __launch_bounds__(256) cost_reduce_kernel(const double* fid, int nfid, const float2* fidff, int nff,
                                                           const double* hp, int nh, double* ring,
                                                           int* t_dev, double* out4, const double* weights, float* bc_next,
                                                           double* gp, double g1, double g2, const NormArgs nprev) {
  // per-thread sums over a fixed stride (FP64 partials in FP64, (hi, lo) pairs as pairs),
  // then one block sum of (hi, lo) pairs
  __shared__ float red[2 * 3 * 32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nfid; i += blockDim.x) s0 += fid[i];
  FF f0 = ff_from_double(s0);
  constexpr int U = 8;  // eight loads in flight, added in index order
  for (int i0 = threadIdx.x; i0 < nff; i0 += U * blockDim.x) {
    float2 pv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      pv[u] = (i < nff) ? fidff[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * (int)blockDim.x < nff) f0 = ff_add(f0, FF{pv[u].x, pv[u].y});
  }
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    s1 += hp[2 * i];
    s2 += hp[2 * i + 1];
  }
  const FF part[3] = {f0, ff_from_double(s1), ff_from_double(s2)};
  double sum[3];
  block_sum_ff<3>(part, red, sum);
  const double a0 = sum[0], a1 = sum[1], a2 = sum[2];
  if (threadIdx.x == 0) {
    if (out4) {  // the three terms and Eq. 8's total L = L_fid + alpha L_A + beta L_Phi, in FP64
      out4[0] = a0;
      out4[1] = a1;
      out4[2] = a2;
      out4[3] = a0 + weights[0] * a1 + weights[1] * a2;
    }
    if (ring) {
      const int t = *t_dev;
      double* r = ring + 3 * (t % kCostRing);
      r[0] = a0;
      r[1] = a1;
      r[2] = a2;
      if (bc_next) {
        *t_dev = t + 1;
        const double p1 = gp[0] * g1, p2 = gp[1] * g2;
        gp[0] = p1;
        gp[1] = p2;
        bc_next[0] = (float)(1.0 / (1.0 - p1));
        bc_next[1] = (float)(1.0 / (1.0 - p2));
      }
    }
  }
  // in update mode, the norms of the previous update (its gather has finished: it precedes this
  // iteration's fork)
  if (bc_next && nprev.part) norms_finalize(nprev.part, nprev.nblk, nprev.pending, nprev.slot, nprev.ring, red);
}

// Running powers gamma^1 and bias corrections 1/(1 - gamma^1) of Eq. 19 for t = 0.
__global__ void init_bias_kernel(float* bc, double* gp, double g1, double g2) {
  if (threadIdx.x != 0) return;
  gp[0] = g1;
  gp[1] = g2;
  bc[0] = (float)(1.0 / (1.0 - g1));
  bc[1] = (float)(1.0 / (1.0 - g2));
}

cudaError_t launch_init_bias(float* bc, double* gp, double g1, double g2, cudaStream_t s) {
  init_bias_kernel<<<1, 32, 0, s>>>(bc, gp, g1, g2);
  return cudaGetLastError();
}

cudaError_t launch_cost_reduce(const double* fid, int nfid, const float2* fidff, int nff, const double* hp, int nh,
                               double* ring, int* t_dev, double* out4, const double* weights, float* bc_next,
                               double* gp, double g1, double g2, const NormArgs& nprev, cudaStream_t s) {
  // 256 threads: 23.4 against 25.4 us per iteration at 64/256/49 with 1024 (the same at 256/1024/225)
  cost_reduce_kernel<<<1, 256, 0, s>>>(fid, nfid, fidff, nff, hp, nh, ring, t_dev, out4, weights, bc_next, gp, g1,
                                        g2, nprev);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Eqs. 16-17 (alpha = beta)
// Per-pixel responses of the 3x3 kernel in FP32, sums of |response| in FP64 in a
// fixed order: block (image k, 16-row chunk) partials, then one ordered pass.
constexpr int kAlphaRows = 16;

int alpha_blocks(int K, int n) { return K * ((n - 2 + kAlphaRows - 1) / kAlphaRows); }

__global__ void __launch_bounds__(256) alpha_partial_kernel(const float* I, int n, int amplitude, double* partial) {
  __shared__ double red[8];
  const int chunks = (n - 2 + kAlphaRows - 1) / kAlphaRows;
  const int k = blockIdx.x / chunks, ch = blockIdx.x - k * chunks;
  const float* img = I + (size_t)k * n * n;
  const int m = n - 2;
  const int y0 = 1 + ch * kAlphaRows, y1 = min(n - 1, y0 + kAlphaRows);
  double acc = 0.0;
  for (int y = y0; y < y1; ++y) {
    for (int x = 1 + threadIdx.x; x <= m; x += 256) {
      float v[3][3];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          float t = img[(y + dy - 1) * n + (x + dx - 1)];
          if (amplitude) t = sqrtf(fmaxf(t, 0.f));
          v[dy][dx] = t;
        }
      // [-1 2 -1; -2 4 -2; -1 2 -1] (Eq. 16)
      const float r = (2.f * v[0][1] - v[0][0] - v[0][2]) + 2.f * (2.f * v[1][1] - v[1][0] - v[1][2]) +
                      (2.f * v[2][1] - v[2][0] - v[2][2]);
      acc += (double)fabsf(r);
    }
  }
  const double s = block_sum_double(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) alpha_final_kernel(const double* partial, int nparts, int K, int n,
                                                          double* weights, double fa, double fb) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += partial[i];
  const double s = block_sum_double(acc, red);
  if (threadIdx.x != 0) return;
  const double m = (double)(n - 2) * (double)(n - 2) * (double)K;
  const double est = 0.2 * sqrt(3.14159265358979323846 / 2.0) * s / m;
  weights[0] = (fa < 0.0) ? est : fa;
  weights[1] = (fb < 0.0) ? est : fb;
}

cudaError_t launch_alpha(const float* I, int K, int n, int amplitude, double* partial, double* weights,
                         double fixed_alpha, double fixed_beta, cudaStream_t s) {
  if (fixed_alpha < 0.0 || fixed_beta < 0.0) {
    const int nb = alpha_blocks(K, n);
    alpha_partial_kernel<<<nb, 256, 0, s>>>(I, n, amplitude, partial);
    alpha_final_kernel<<<1, 256, 0, s>>>(partial, nb, K, n, weights, fixed_alpha, fixed_beta);
  } else {
    alpha_final_kernel<<<1, 256, 0, s>>>(partial, 0, K, n, weights, fixed_alpha, fixed_beta);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Sec. 6.3 scaling maps
// The measured side of the residual g(|o|^2) - g(max(I, 0)) of Eq. 4 (g = sqrt) and of the Sec. 6.3
// maps, mapped once per set of measurements.
__global__ void gmap_kernel(const float4* __restrict__ I, float4* __restrict__ Ig, size_t n4, int fidelity,
                            float gexp) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    float4 v = I[i];
    float* e = reinterpret_cast<float*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float x = fmaxf(e[j], 0.f);
      e[j] = (fidelity == 1) ? sqrtf(x) : (fidelity == 2) ? powf(x, gexp) : log1pf(x);
    }
    Ig[i] = v;
  }
}

__global__ void gmap_tail_kernel(const float* I, float* Ig, size_t b, size_t count, int fidelity, float gexp) {
  const size_t i = b + threadIdx.x;
  if (i >= count) return;
  const float x = fmaxf(I[i], 0.f);
  Ig[i] = (fidelity == 1) ? sqrtf(x) : (fidelity == 2) ? powf(x, gexp) : log1pf(x);
}

cudaError_t launch_gmap(const float* I, float* Ig, size_t count, int fidelity, float gexp, cudaStream_t s) {
  // I and Ig come from cudaMalloc (256-byte aligned); the last count % 4 elements go one by one
  const size_t n4 = count / 4;
  if (n4) {
    const int blocks = (int)std::min<size_t>((n4 + 255) / 256, 152 * 8);
    gmap_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4*>(I), reinterpret_cast<float4*>(Ig), n4,
                                       fidelity, gexp);
  }
  if (count % 4) gmap_tail_kernel<<<1, 32, 0, s>>>(I, Ig, n4 * 4, count, fidelity, gexp);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ initial state
__global__ void init_small_kernel(const float* Ic, float2* small, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n * n) return;
  const int y = j / n, x = j - y * n;
  const float a = sqrtf(fmaxf(Ic[j], 0.f));
  small[j] = make_float2(((x + y) & 1) ? -a : a, 0.f);  // (-1)^(x+y): fftshift of the DFT
}

cudaError_t launch_init_small(const float* I_c, float2* small, int n, cudaStream_t s) {
  init_small_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(I_c, small, n);
  return cudaGetLastError();
}

__global__ void embed_kernel(const float2* small, float2* psi, int n, int N, int oy, int ox, float gain) {
  const size_t total = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / N), x = (int)(i - (size_t)y * N);
    const int jy = y - oy, jx = x - ox;
    float2 v = make_float2(0.f, 0.f);
    if (jy > 0 && jy < n && jx > 0 && jx < n) v = cscale(small[jy * n + jx], gain);  // Nyquist row/col zeroed
    psi[i] = v;
  }
}

cudaError_t launch_embed(const float2* small, float2* psi, int n, int N, int oy, int ox, float gain, cudaStream_t s) {
  embed_kernel<<<1024, 256, 0, s>>>(small, psi, n, N, oy, ox, gain);
  return cudaGetLastError();
}

__global__ void fill_f2_kernel(float2* p, size_t count, float2 v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void fill_f_kernel(float* p, size_t count, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

cudaError_t launch_fill_f2(float2* p, size_t count, float2 value, cudaStream_t s) {
  fill_f2_kernel<<<1024, 256, 0, s>>>(p, count, value);
  return cudaGetLastError();
}
cudaError_t launch_fill_f(float* p, size_t count, float value, cudaStream_t s) {
  fill_f_kernel<<<1024, 256, 0, s>>>(p, count, value);
  return cudaGetLastError();
}

__global__ void support_pupil_kernel(float2* p, const int* sidx_map, int nn) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nn) p[j] = make_float2(sidx_map[j] >= 0 ? 1.f : 0.f, 0.f);
}

cudaError_t launch_support_pupil(float2* p, const int* sidx_map, int n, cudaStream_t s) {
  support_pupil_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(p, sidx_map, n * n);
  return cudaGetLastError();
}

__global__ void count_nonfinite_kernel(const float* x, size_t count, int* flag) {
  int bad = 0;
  const size_t n4 = count / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);  // cudaMalloc'd: 16-byte aligned
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = x4[i];
    bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
  }
  for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) *flag = 1;
}

cudaError_t launch_count_nonfinite(const float* x, size_t count, int* flag, cudaStream_t s) {
  count_nonfinite_kernel<<<4 * 152, 256, 0, s>>>(x, count, flag);
  return cudaGetLastError();
}

}  // namespace elf
