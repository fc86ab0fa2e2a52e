// Internal interfaces between the host API (elfpie_api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

namespace elf {

// ---------------------------------------------------------------- programmatic dependent launch
// A chain of kernels on one stream: each kernel lets the next be launched once all its CTAs have
// started (pdl_launch_dependents), so that the next kernel's CTAs take the SMs it frees and run their
// independent prologue; the next kernel waits (pdl_wait) for its completion, with its memory visible,
// before reading what it wrote.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch of a kernel that may start while the previous kernel of the stream still runs (it calls
// pdl_wait before reading that kernel's results).  The previous operation on the stream must be a
// kernel launch (no event in between).
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

constexpr int kGatherSeg = 64;    // row segment of the gather lists (two pixels per thread)
inline int gather_seg(int N) { return N < kGatherSeg ? N : kGatherSeg; }
constexpr int kCostRing = 4096;   // iterations kept in the cost ring buffer
constexpr int kGraphIters = 8;    // iterations per graph launch of elf_step when tracing is off (even)

// ---------------------------------------------------------------- tile kernel
// One cluster of CS CTAs per LED runs Eqs. 1, 5/4, 12, 11/10 and F_B^H of Eq. 9.
struct TileArgs {
  const float2* psi;      // N x N centred spectrum
  const float2* pupil;    // n x n centred pupil (read on the support only)
  const float* meas;      // K x n x n measured intensities (gradient mode)
  const int2* origin;     // K crop origins (.x = row, .y = col)
  const int* row_xs;      // n: first support column of each pupil row (or 0)
  const int* row_cnt;     // n: support pixels in each pupil row
  const int* row_off;     // n: compact index of the first support pixel of each row
  const float2* tw;       // n team twiddles tw[k1 * Q + l] = e^{-2 pi i l k1 / n}
  float2* G;              // K x S tile gradients on the support (gradient mode)
  float2* cost_ff;        // K x CS fidelity cost partials (one per CTA), (hi, lo) float pairs
  int* err;               // set to 1 when a bounded wait of a DSMEM exchange ran out
  float* I_out;           // K x n x n predicted intensities (simulate mode)
  int N, K, S, Blo, nb, rowsA;
  float scale;            // 1 / (u^2 n^2)
  float tau, eta;
  float gexp;             // gamma of the power map (fidelity 2)
  int fidelity, iso;      // fidelity 1-3 read meas = g(max(I, 0)): sqrt (Eq. 4) or a Sec. 6.3 map
  int mode;               // 0 = gradient, 1 = simulate |o|^2, 2 = gradient of multiplexed images:
                          // meas holds the per-image factor f (mux_kernels.cu), W = o f
  int mux;                // M: LEDs per image; LED k reads image k / M in mode 2
  int led0, nled;         // LEDs [led0, led0 + nled) (nled = 0: all K from LED 0)
};
int tile_cluster_size(int n);
int tile_warps(int n);                        // warps per CTA of the tile kernel
size_t tile_smem_bytes(int n, int cs, int rowsA);
cudaError_t prepare_tile(int n, int rowsA);   // sets kernel attributes; call outside capture
cudaError_t launch_tile(const TileArgs& a, int n, cudaStream_t s);

// ---------------------------------------------------------------- split tile path (tile_split.cu)
// The same tile work as three kernels (inverse rows, columns + stencil, forward rows) with the support
// band of each LED in device memory: band_in / band_out hold K x nb x n complex each.  Gradient mode only.
bool tile_split_selected(int n, int mux, int tile_dft, int tile_path);
cudaError_t prepare_tile_split(int n);        // sets kernel attributes; call outside capture
cudaError_t launch_tile_split(const TileArgs& a, int n, float2* band_in, float2* band_out, cudaStream_t s);

// ---------------------------------------------------------------- multiplexed images (mux_kernels.cu)
int mux_blocks_per_image(int n);  // cost partials per image of mux_omega
cudaError_t launch_mux_resid(const float* Imod, const float* meas, float* R, float* F, int n_img, int M, int n,
                             int fidelity, float gexp, float eta, cudaStream_t s);
cudaError_t launch_mux_omega(const float* R, float* F, double* partial, int n_img, int n, float tau, int iso,
                             cudaStream_t s);
cudaError_t launch_mux_sum(const float* Imod, float* out, int n_img, int M, int n, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core tile path (tc_dft.cu)
constexpr int kTcN = 128;     // tile side of the tensor-core path
constexpr int kTcBand = 64;   // padded band of support rows / columns
// BF16 hi/lo operand images (tc_dft.cu): R rows x KR real K take R * KR * 4 bytes
constexpr size_t kTcImgX = (size_t)kTcBand * 2 * kTcBand * 4;  // X: 64 rows, K = 128
constexpr size_t kTcImgY = (size_t)kTcN * 2 * kTcBand * 4;     // Y' (and one gemm-1 A): 128 rows, K = 128
constexpr size_t kTcImgW = (size_t)kTcN * 2 * kTcN * 4;        // W' (and one gemm-3 A): 128 rows, K = 256
constexpr size_t kTcImgZ = (size_t)kTcN * 2 * kTcN * 4;        // Z: 128 rows (64 used), K = 256
struct TcArgs {
  const float2* psi; const float2* pupil; const int2* origin;
  const int* row_xs; const int* row_cnt; const int* row_off;
  const float* meas;
  const unsigned char *cA1, *cB2, *cA3, *cB4;  // constant operand images (tc_constant_image 0..3)
  unsigned char *iX, *iY, *iW, *iZ;           // per-LED data operand images
  float2* Ot;           // per-LED O' = transposed raw IDFT (128 x 128)
  float2* G;            // K x S output on the support
  double* costpart;     // K fidelity cost partials
  int* err;             // set when a bounded wait runs out
  int n, N, K, S, Blo, nb;
  float scale, tau, eta, gexp;
  int fidelity, iso;      // fidelity 1-3 read meas = g(max(I, 0)): sqrt (Eq. 4) or a Sec. 6.3 map
};
// Constant operand images, built on the host in FP64 and split into BF16 hi + lo:
// 0 = gemm 1's two A, 1 = gemm 2's B, 2 = gemm 3's two A, 3 = gemm 4's B.
std::vector<unsigned char> tc_constant_image(int which, int Blo, int nb);
cudaError_t prepare_tc();
cudaError_t launch_tc_tile(const TcArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- FFT layout (see fft.cuh)
// lanes per transform Q, and the padded buffer length L + L / Q
inline int fft_team_lanes(int L) {
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  return 1 << (lg / 2);
}
inline int fft_padded_length(int L) { return L + L / fft_team_lanes(L); }

// ---------------------------------------------------------------- big FFTs
// 2D transforms of an L x L array: rows pass then columns pass, unnormalised.
cudaError_t prepare_fft(int L);               // sets kernel attributes; call outside capture
// src != null: the input is read from src and the result written to data (src is not modified).
// tmp != null (an L x L scratch array, L >= 512): the column transform runs as the two register passes
// of the four-step split instead of the shared-memory strip kernel.
// pdl: the passes are chained by programmatic dependent launch (dep: the rows pass too, which then
// directly follows another kernel of the stream).
cudaError_t launch_fft2(float2* data, int L, bool inverse, const float2* tw, cudaStream_t s,
                        const float2* src = nullptr, float2* tmp = nullptr, bool dep = false, bool pdl = true);
// dst[y][x] = (-1)^(x+y) * scale * src[y][x] over an L x L array (src may equal dst).
cudaError_t launch_sign_scale(const float2* src, float2* dst, int L, float scale, cudaStream_t s);

// ---------------------------------------------------------------- Hessian branch
struct HessArgs {
  const float2* ot;       // unnormalised IDFT_N(Psi) (no shift applied)
  float2* q;              // out: (-1)^(x+y) q / A, ready for the forward DFT
  double* costpart;       // [blocks][2] (L_A, L_Phi) partials
  const double* weights;  // device [alpha, beta]
  int N;
  float invA, tau, eta;
  int iso;
};
int hess_blocks(int N);
// pdl: launched as a programmatic dependent of the column pass it follows on the stream.
cudaError_t launch_hessian(const HessArgs& a, cudaStream_t s, bool pdl);

// ---------------------------------------------------------------- gather + AdaBelief
struct GatherArgs {
  const float2* G;        // K x S
  const float2* pupil;    // n x n
  const int2* origin;     // K
  const int* row_xs; const int* row_cnt; const int* row_off;
  const int* seg_ptr;     // N * tiles_x + 1 offsets of the lists per (row, 32-pixel segment)
  const int4* seg_ent;    // entries, ascending LED: {LED, compact G row offset - first x, pupil index - x,
                          // first x | count << 16}
  const float2* gH;       // N x N Hessian gradient (may be null)
  const float2* psi;      // Psi^t
  float2* psi_out;        // Psi^(t+1) (update mode; another buffer than psi)
  float2* mu; float* v; float* delta;   // state (update mode, in place)
  float2* g_out;          // gradient output (gradient mode)
  const float* bc;        // Eq. 19 bias corrections 1/(1-g1^t), 1/(1-g2^t) of this iteration
  int N, n, S, K, tiles_x;
  float g1, g2, eta;
  int mode;               // 0 = AdaBelief update, 1 = write g
  // update mode: this block's sums of |g|^2 and |Delta|^2 into norm_part[block] (the buffer of this
  // iteration's parity, gather_blocks(N) entries), and *norm_pending = 1
  float2* norm_part;
  int* norm_pending;
};
int gather_blocks(int N);
// The norms (||g||, ||Delta Psi||) of an update from its gather's partials: part [nblk], added in block
// order when *pending, into ring [kCostRing][2] at slot *slot % kCostRing; then *slot += 1, *pending = 0.
struct NormArgs {
  const float2* part;
  int nblk;
  int* pending;
  int* slot;
  double* ring;
};
cudaError_t launch_norms_finalize(const NormArgs& n, cudaStream_t s);
// A wait that runs out on purpose (peak.cu): sets *err after `limit` polls of a barrier nothing completes.
cudaError_t launch_wait_timeout(int* err, long long limit, cudaStream_t s);
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- pupil
struct PupilArgs {
  const float2* G; const float2* psi; const int2* origin;
  const int* sup_y; const int* sup_x; const int* sidx_map;   // S, S, n*n
  float2* part;           // Q x S
  int* done;              // ceil(S / 256) counters of finished chunks, zero between launches
  const float2* pupil;    // P^t
  float2* pupil_next;     // P^{t+1}
  float2* mu; float* v; float* delta;
  float2* g_out;          // gradient mode output (n x n)
  const float* bc;        // Eq. 19 bias corrections of this iteration
  int N, n, S, K, Q, filter;
  float w0, w1;           // 1D Gaussian weights (centre, side), normalised
  float g1, g2, eta;
  int mode;               // 0 = update, 1 = write g
};
int pupil_chunks(int K, int S);
cudaError_t launch_pupil_partial(const PupilArgs& a, cudaStream_t s);
cudaError_t launch_pupil_offsupport(const PupilArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- reductions / setup
// out4 != null: (L_fid, L_A, L_Phi, L) with L = L_fid + weights[0] L_A + weights[1] L_Phi (Eq. 8).
// bc_next != null (with ring): also t += 1, gp *= gamma and bc_next = the next iteration's corrections.
cudaError_t launch_cost_reduce(const double* fid, int nfid, const float2* fidff, int nff, const double* hp, int nh,
                               double* ring, int* t_dev, double* out4, const double* weights, float* bc_next,
                               double* gp, double g1, double g2, const NormArgs& nprev,
                               cudaStream_t s);
cudaError_t launch_init_bias(float* bc, double* gp, double g1, double g2, cudaStream_t s);
int alpha_blocks(int K, int n);
cudaError_t launch_alpha(const float* I, int K, int n, int amplitude, double* partial, double* weights,
                         double fixed_alpha, double fixed_beta, cudaStream_t s);
// Ig = g(max(I, 0)), the measured side of the residual (fidelity 1: sqrt, Eq. 4; 2: x^gexp, 3: ln(x + 1),
// Sec. 6.3)
cudaError_t launch_gmap(const float* I, float* Ig, size_t count, int fidelity, float gexp, cudaStream_t s);
cudaError_t launch_init_small(const float* I_c, float2* small, int n, cudaStream_t s);
cudaError_t launch_embed(const float2* small, float2* psi, int n, int N, int oy, int ox, float gain,
                         cudaStream_t s);
cudaError_t launch_fill_f2(float2* p, size_t count, float2 value, cudaStream_t s);
cudaError_t launch_fill_f(float* p, size_t count, float value, cudaStream_t s);
cudaError_t launch_support_pupil(float2* p, const int* sidx_map, int n, cudaStream_t s);
cudaError_t launch_count_nonfinite(const float* x, size_t count, int* flag, cudaStream_t s);

}  // namespace elf
