// Host side of the C ABI declared in include/elfpie.h.
//
// elf_create validates the geometry of Sec. 3.1 (LED offsets, crop windows,
// pupil support), builds the lookup tables the kernels use (support runs per
// pupil row, compact support order, per-spectrum-tile LED lists for the
// deterministic gather of Eq. 9) and allocates every device buffer once.
// One iteration of Algorithm 1 is the launch sequence in enqueue_iteration; for
// elf_step it is captured once into a CUDA graph whose Hessian branch
// (Eqs. 6-7, 13-14) runs on a second stream concurrently with the tile kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/elfpie.h"
#include "internal.cuh"

using namespace elf;

namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define ELF_CK(call)                                                                               \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return set_error(e_ == cudaErrorMemoryAllocation ? ELF_ENOMEM : ELF_ECUDA,                   \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

double round_half_away(double x) { return (x < 0 ? -1.0 : 1.0) * std::floor(std::fabs(x) + 0.5); }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

namespace elf {
// error reporting for the entry points defined in other translation units
int noalloc_set_error(int code, const char* msg) { return set_error(code, msg); }
}  // namespace elf

struct elf_handle_s {
  int n = 0, u = 0, N = 0, K = 0, S = 0, Blo = 0, nb = 0, rowsA = 0, cs = 1, Q = 1;
  int hblocks = 0, tiles_x = 0, centre = 0;
  int mux = 1, n_img = 0;  // LEDs per measured image (Eq. 1) and the number of images K / mux
  double dk = 0.0;
  double pupil_cut = 0.0;  // NA / lambda, the pupil radius in cycles/um
  elf_options opt{};
  cudaStream_t user = nullptr, cap = nullptr, aux = nullptr, paux = nullptr;  // paux: pupil chain
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tile = nullptr, ev_cost = nullptr,
              ev_pu = nullptr;
  bool have_meas = false;
  bool tracing = false;
  bool shard_open = false;  // elf_shard_tiles ran; elf_shard_finish has not
  bool split = false;       // the tile work runs as the three split kernels (tile_split.cu)
  float2 *band_in = nullptr, *band_out = nullptr;  // their K x nb x n support bands
  int shard_k0 = 0, shard_k1 = 0;
  int graph_kernels = 0;
  cudaEvent_t ev_stage[2 * ELF_NSTAGES] = {};
  cudaGraphExec_t graph[2] = {};  // iteration from psi_buf[p] into psi_buf[p ^ 1]
  cudaGraphExec_t graph_r[2] = {};  // kGraphIters iterations from buffer p back to buffer p (untraced)
  std::vector<int2> origin_h;
  std::vector<int> sidx_h;  // linear support indices in compact order
  float gw0 = 0.f, gw1 = 0.f;
  // device tables
  int2* origin = nullptr;
  int *row_xs = nullptr, *row_cnt = nullptr, *row_off = nullptr;
  int *sup_y = nullptr, *sup_x = nullptr, *sidx_map = nullptr;
  int* seg_ptr = nullptr;   // gather lists per (row, 32-pixel segment), CSR offsets
  int4* seg_ent = nullptr;  // their entries
  float2 *tw_n = nullptr, *tw_N = nullptr;
  // data and state
  float* I = nullptr;
  float* Ig = nullptr;  // g(max(I, 0)): sqrt (fidelity 1) or a Sec. 6.3 map (2, 3); null for fidelity 0
  // multiplexed images (mux > 1): per-LED |o|^2, per-image residual and factor f, cost partials
  float* Imod = nullptr;
  float* mux_r = nullptr;
  float* mux_f = nullptr;
  double* mux_cost = nullptr;
  // Psi is double-buffered: an iteration reads psi_buf[cur] and its gather writes Psi^(t+1) into the
  // other buffer, so that the Eq. 18 partials (which read Psi^t) need not finish before the gather;
  // psi always points at the current buffer
  float2* psi_buf[2] = {};
  int cur = 0;
  float2 *psi = nullptr, *mu_psi = nullptr;
  float *v_psi = nullptr, *delta_psi = nullptr;
  // P is double-buffered like Psi (the Eq. 19 update writes P^(t+1) into the other buffer); with
  // learn_pupil = 0 both iterations read pupil_buf[0].  pupil always points at the current buffer.
  float2* pupil_buf[2] = {};
  float2 *pupil = nullptr, *mu_p = nullptr;
  float *v_p = nullptr, *delta_p = nullptr;
  // scratch
  float2 *G = nullptr, *ot = nullptr, *q = nullptr, *small = nullptr, *part = nullptr;
  float2* fft_tmp = nullptr;  // scratch of the N x N transforms (four-step column passes), N >= 512
  int* pdone = nullptr;  // per 256 support pixels: Eq. 18 chunks finished (reset by the partial kernel)
  float2 *psi_eval = nullptr, *pupil_eval = nullptr, *g_psi = nullptr, *g_p = nullptr, *pupil_unit = nullptr;
  float2* cost_ff = nullptr;  // per-warp (hi, lo) fidelity cost partials of the tile kernel
  double *cost_fid = nullptr, *cost_h = nullptr, *ring = nullptr, *weights = nullptr, *alpha_part = nullptr,
         *out4 = nullptr;
  int *t_dev = nullptr, *flag = nullptr;
  float2* norm_part = nullptr;  // [2 parities][gather blocks] sums of |g|^2 and |Delta|^2
  double* norm_ring = nullptr;  // [kCostRing][2] (||g||, ||Delta Psi||)
  int* norm_state = nullptr;    // [0], [1] partials of parity 0 / 1 pending; [2] next ring slot
  size_t device_bytes = 0;  // sum of this handle's device allocations
  // tensor-core tile path (tile_dft = 1)
  unsigned char *tc_iX = nullptr, *tc_iY = nullptr, *tc_iW = nullptr, *tc_iZ = nullptr;  // operand images
  unsigned char* tc_c[4] = {nullptr, nullptr, nullptr, nullptr};                       // constant images
  float2* tc_Ot = nullptr;
  int* tc_err = nullptr;  // device error flag of the bounded waits (tile exchanges, tensor-core path)
  float* bc = nullptr;   // Eq. 19 bias corrections, per buffer parity: bc[2p, 2p + 1] for the iteration
                         // that reads psi_buf[p] (the iteration writes the pair of the other parity)
  double* gp = nullptr;  // (gamma1^(t+1), gamma2^(t+1)) for the next iteration
  std::vector<void*> allocs;
};

namespace {

template <typename T>
int dalloc(elf_handle h, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess)
    return set_error(e == cudaErrorMemoryAllocation ? ELF_ENOMEM : ELF_ECUDA,
                     std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(v);
  h->device_bytes += count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  *p = static_cast<T*>(v);
  return ELF_OK;
}

template <typename T>
int upload(elf_handle h, T** p, const std::vector<T>& v) {
  int rc = dalloc(h, p, v.size());
  if (rc) return rc;
  if (!v.empty()) ELF_CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ELF_OK;
}

// Team twiddles of a length-L transform (fft.cuh): tw[k1 * Q + l] = e^{-2 pi i l k1 / L},
// computed in FP64.
std::vector<float2> twiddles(int L) {
  const int Q = fft_team_lanes(L), P = L / Q;
  std::vector<float2> t(L);
  const double pi = 3.14159265358979323846;
  for (int k1 = 0; k1 < P; ++k1)
    for (int l = 0; l < Q; ++l) {
      const double a = -2.0 * pi * (double)((long)l * k1 % L) / (double)L;
      t[k1 * Q + l] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  return t;
}

// Timing event of a stage boundary (recorded into the graph when tracing is on).
int mark(elf_handle h, cudaStream_t s, int stage, int end) {
  if (!h->tracing) return ELF_OK;
  ELF_CK(cudaEventRecordWithFlags(h->ev_stage[2 * stage + end], s, cudaEventRecordExternal));
  return ELF_OK;
}

#define ELF_MARK(s, stage, end)                          \
  do {                                                   \
    if (int rc_ = mark(h, (s), (stage), (end))) return rc_; \
  } while (0)

// Parts of one iteration (enqueue_iteration): the front part forks the Hessian branch and the
// off-support pupil update onto the auxiliary stream and runs the tile kernel for LEDs
// [led_begin, led_end) on s0; the back part (every LED's tile results present) runs the Eq. 8 cost
// reduction, the pupil chain and the gather, and joins the streams into s0.
enum { kPartFront = 1, kPartBack = 2, kPartAll = 3 };

// One outer iteration of Algorithm 1 (mode 0) or a gradient evaluation (mode 1).
// In mode 0 the gather writes Psi^(t+1) into psi_out (not psi, which the pupil chain still reads)
// and the pupil update writes P^(t+1) into pupil_out (not pupil, which the gather still reads).
// parts selects the front and / or back part; the tile kernel covers LEDs [led_begin, led_end).
int enqueue_iteration(elf_handle h, int mode, cudaStream_t s0, const float2* psi, const float2* pupil,
                      float2* psi_out, float2* pupil_out, int parts = kPartAll, int led_begin = 0, int led_end = -1) {
  const bool pupil_path = (mode == 1) || h->opt.learn_pupil;
  const size_t A = (size_t)h->N * h->N;
  if (led_end < 0) led_end = h->K;
  // Eq. 19 bias corrections of this iteration and of the next (double-buffered with Psi)
  const int par = (psi == h->psi_buf[1]) ? 1 : 0;
  float* bc_cur = h->bc + 2 * par;
  float* bc_next = h->bc + 2 * (par ^ 1);
  PupilArgs pa{};
  pa.G = h->G;
  pa.psi = psi;
  pa.origin = h->origin;
  pa.sup_y = h->sup_y;
  pa.sup_x = h->sup_x;
  pa.sidx_map = h->sidx_map;
  pa.part = h->part;
  pa.pupil = pupil;
  pa.pupil_next = pupil_out;
  pa.mu = h->mu_p;
  pa.v = h->v_p;
  pa.delta = h->delta_p;
  pa.g_out = h->g_p;
  pa.bc = bc_cur;
  pa.N = h->N;
  pa.n = h->n;
  pa.S = h->S;
  pa.K = h->K;
  pa.Q = h->Q;
  pa.filter = h->opt.pupil_filter;
  pa.w0 = h->gw0;
  pa.w1 = h->gw1;
  pa.g1 = (float)h->opt.gamma1;
  pa.g2 = (float)h->opt.gamma2;
  pa.eta = (float)h->opt.eta_opt;
  pa.mode = mode;
  pa.done = h->pdone;
  GatherArgs ga{};
  ga.G = h->G;
  ga.pupil = pupil;
  ga.origin = h->origin;
  ga.row_xs = h->row_xs;
  ga.row_cnt = h->row_cnt;
  ga.row_off = h->row_off;
  ga.seg_ptr = h->seg_ptr;
  ga.seg_ent = h->seg_ent;
  ga.gH = h->q;
  ga.psi = psi;
  ga.psi_out = psi_out;
  ga.mu = h->mu_psi;
  ga.v = h->v_psi;
  ga.delta = h->delta_psi;
  ga.g_out = h->g_psi;
  ga.bc = bc_cur;
  ga.N = h->N;
  ga.n = h->n;
  ga.S = h->S;
  ga.K = h->K;
  ga.tiles_x = h->tiles_x;
  ga.g1 = (float)h->opt.gamma1;
  ga.g2 = (float)h->opt.gamma2;
  ga.eta = (float)h->opt.eta_opt;
  ga.mode = mode;
  const int nblk = gather_blocks(h->N);
  ga.norm_part = h->norm_part + (size_t)par * nblk;
  ga.norm_pending = h->norm_state + par;
  if (parts & kPartFront) {
    ELF_MARK(s0, ELF_STAGE_ITERATION, 0);
    // Hessian branch on the auxiliary stream: O, Eqs. 6-7 and 13-14, F_A^H
    ELF_CK(cudaEventRecord(h->ev_fork, s0));
    ELF_CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    ELF_MARK(h->aux, ELF_STAGE_HESSIAN, 0);
    // the branch's kernels chained by programmatic dependent launch only where the branch is the longer
    // one (N <= 256: 27.3 against 29.5 us per iteration at 64/256/49); beside long tile work the early
    // CTAs of the high-priority branch would wait on SMs the tile kernels need (0.172 against 0.163 ms
    // at 256/1024/225)
    const bool hpdl = h->N <= 256;
    ELF_CK(launch_fft2(h->ot, h->N, true, h->tw_N, h->aux, psi, h->fft_tmp, false, hpdl));  // the first pass reads Psi
    HessArgs ha{};
    ha.ot = h->ot;
    ha.q = h->q;
    ha.costpart = h->cost_h;
    ha.weights = h->weights;
    ha.N = h->N;
    ha.invA = (float)(1.0 / (double)A);
    ha.tau = (float)h->opt.tau_h;
    ha.eta = (float)h->opt.eta_h;
    ha.iso = h->opt.omega_iso;
    ELF_CK(launch_hessian(ha, h->aux, hpdl));
    ELF_CK(launch_fft2(h->q, h->N, false, h->tw_N, h->aux, nullptr, h->fft_tmp, true, hpdl));  // follows the stencil
    ELF_MARK(h->aux, ELF_STAGE_HESSIAN, 1);
    ELF_CK(cudaEventRecord(h->ev_join, h->aux));

    // Eq. 19 off the support (gradient 0) needs nothing from the tile kernel: it runs on the auxiliary
    // stream after the Hessian branch, on the SMs the tile work leaves free (measured against the pupil
    // stream after the Hessian branch: 0.1680 against 0.1693 ms per iteration at 256/1024/225, 0.0532
    // against 0.0564 ms at 128/512/225)
    if (pupil_path) {
      ELF_MARK(h->aux, ELF_STAGE_PUPIL_UPDATE, 0);
      ELF_CK(launch_pupil_offsupport(pa, h->aux));
      ELF_MARK(h->aux, ELF_STAGE_PUPIL_UPDATE, 1);
    }

    // tile path: Eqs. 1, 5 (4), 12, 11 (10) and F_B^H of Eq. 9
    TileArgs ta{};
    ta.psi = psi;
    ta.pupil = pupil;
    ta.meas = h->opt.fidelity >= 1 ? h->Ig : h->I;
    ta.origin = h->origin;
    ta.row_xs = h->row_xs;
    ta.row_cnt = h->row_cnt;
    ta.row_off = h->row_off;
    ta.tw = h->tw_n;
    ta.G = h->G;
    ta.cost_ff = h->cost_ff;
    ta.err = h->tc_err;
    ta.I_out = nullptr;
    ta.N = h->N;
    ta.K = h->K;
    ta.S = h->S;
    ta.Blo = h->Blo;
    ta.nb = h->nb;
    ta.rowsA = h->rowsA;
    ta.scale = (float)(1.0 / ((double)h->u * h->u * (double)h->n * h->n));
    ta.tau = (float)h->opt.tau_fid;
    ta.eta = (float)h->opt.eta_h;
    ta.gexp = (float)h->opt.g_exponent;
    ta.fidelity = h->opt.fidelity;
    ta.iso = h->opt.omega_iso;
    ta.mode = 0;
    ta.mux = h->mux;
    ta.led0 = led_begin;
    ta.nled = led_end - led_begin;
    ELF_MARK(s0, ELF_STAGE_TILE, 0);
    if (h->opt.tile_dft) {
      TcArgs tc{};
      tc.psi = psi;
      tc.pupil = pupil;
      tc.origin = h->origin;
      tc.row_xs = h->row_xs;
      tc.row_cnt = h->row_cnt;
      tc.row_off = h->row_off;
      tc.meas = ta.meas;
      tc.cA1 = h->tc_c[0];
      tc.cB2 = h->tc_c[1];
      tc.cA3 = h->tc_c[2];
      tc.cB4 = h->tc_c[3];
      tc.iX = h->tc_iX;
      tc.iY = h->tc_iY;
      tc.iW = h->tc_iW;
      tc.iZ = h->tc_iZ;
      tc.Ot = h->tc_Ot;
      tc.G = h->G;
      tc.costpart = h->cost_fid;
      tc.err = h->tc_err;
      tc.n = h->n;
      tc.N = h->N;
      tc.K = h->K;
      tc.S = h->S;
      tc.Blo = h->Blo;
      tc.nb = h->nb;
      tc.scale = ta.scale;
      tc.tau = ta.tau;
      tc.eta = ta.eta;
      tc.gexp = ta.gexp;
      tc.fidelity = ta.fidelity;
      tc.iso = ta.iso;
      ELF_CK(launch_tc_tile(tc, s0));
    } else if (h->mux > 1) {
      // multiplexed images: |o|^2 of every LED, per-image residual / normaliser / factor f, then
      // W = o f per LED (mux_kernels.cu)
      TileArgs t1 = ta;
      t1.mode = 1;
      t1.I_out = h->Imod;
      ELF_CK(launch_tile(t1, h->n, s0));
      ELF_CK(launch_mux_resid(h->Imod, ta.meas, h->mux_r, h->mux_f, h->n_img, h->mux, h->n, h->opt.fidelity, ta.gexp,
                              ta.eta, s0));
      ELF_CK(launch_mux_omega(h->mux_r, h->mux_f, h->mux_cost, h->n_img, h->n, ta.tau, ta.iso, s0));
      TileArgs t2 = ta;
      t2.mode = 2;
      t2.meas = h->mux_f;
      ELF_CK(launch_tile(t2, h->n, s0));
    } else if (ta.nled > 0 && h->split) {
      ELF_CK(launch_tile_split(ta, h->n, h->band_in, h->band_out, s0));
    } else if (ta.nled > 0) {
      ELF_CK(launch_tile(ta, h->n, s0));
    }
    ELF_MARK(s0, ELF_STAGE_TILE, 1);
  }  // front part
  if (!(parts & kPartBack)) return ELF_OK;

  // Eq. 8 costs on the auxiliary stream once the Hessian partials (same stream) and the tile
  // kernel's partials exist, beside the gather and pupil kernels below
  ELF_CK(cudaEventRecord(h->ev_tile, s0));
  ELF_CK(cudaStreamWaitEvent(h->aux, h->ev_tile, 0));
  ELF_MARK(h->aux, ELF_STAGE_COST, 0);
  {
    // fidelity partials: FP64 per LED (tensor-core path), per image block (multiplexed images), or
    // the tile kernel's per-CTA pairs
    const bool tc = h->opt.tile_dft != 0, mx = h->mux > 1;
    const double* fid = mx ? h->mux_cost : h->cost_fid;
    const int nfid = tc ? h->K : (mx ? h->n_img * mux_blocks_per_image(h->n) : 0);
    // in update mode it also closes the iteration (t, running powers, the next bias corrections)
    ELF_CK(launch_cost_reduce(fid, nfid, h->cost_ff, (tc || mx) ? 0 : h->K * h->cs, h->cost_h,
                              h->hblocks, mode == 0 ? h->ring : nullptr, h->t_dev, mode == 1 ? h->out4 : nullptr,
                              h->weights, mode == 0 ? bc_next : nullptr, h->gp, h->opt.gamma1, h->opt.gamma2,
                              NormArgs{h->norm_part + (size_t)(par ^ 1) * nblk, nblk, h->norm_state + (par ^ 1),
                                       h->norm_state + 2, h->norm_ring},
                              h->aux));
  }
  ELF_MARK(h->aux, ELF_STAGE_COST, 1);
  ELF_CK(cudaEventRecord(h->ev_cost, h->aux));

  // the pupil chain on its own stream, beside the gather: the Eq. 18 partials, whose last blocks
  // apply Eq. 19 on the support (Eq. 19 off the support ran on the auxiliary stream after the
  // Hessian branch).  The partials read Psi^t, which the gather leaves in place (it writes
  // Psi^(t+1) into the other buffer)
  if (pupil_path) {
    ELF_CK(cudaStreamWaitEvent(h->paux, h->ev_tile, 0));
    ELF_MARK(h->paux, ELF_STAGE_PUPIL_GRAD, 0);
    ELF_CK(launch_pupil_partial(pa, h->paux));
    ELF_MARK(h->paux, ELF_STAGE_PUPIL_GRAD, 1);
    ELF_CK(cudaEventRecord(h->ev_pu, h->paux));
  }

  ELF_CK(cudaStreamWaitEvent(s0, h->ev_join, 0));
  ELF_MARK(s0, ELF_STAGE_GATHER, 0);
  ELF_CK(launch_gather(ga, s0));
  ELF_MARK(s0, ELF_STAGE_GATHER, 1);
  if (pupil_path) ELF_CK(cudaStreamWaitEvent(s0, h->ev_pu, 0));  // the pupil chain joins the iteration
  // the cost reduction (which also closed the iteration) joins it
  ELF_CK(cudaStreamWaitEvent(s0, h->ev_cost, 0));
  ELF_MARK(s0, ELF_STAGE_ITERATION, 1);
  return ELF_OK;
}

// Captures `iters` iterations starting from buffer p into one executable graph.
int capture_iterations(elf_handle h, int p, int iters, cudaGraphExec_t* out, int* kernels) {
  cudaGraph_t g = nullptr;
  ELF_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  const bool lp = h->opt.learn_pupil != 0;
  int rc = ELF_OK;
  for (int i = 0; i < iters && rc == ELF_OK; ++i) {
    const int q = p ^ (i & 1);  // buffers alternate iteration by iteration
    rc = enqueue_iteration(h, 0, h->cap, h->psi_buf[q], h->pupil_buf[lp ? q : 0], h->psi_buf[q ^ 1],
                           lp ? h->pupil_buf[q ^ 1] : nullptr);
  }
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  if (rc != ELF_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return set_error(ELF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (kernels) {
    size_t nn = 0;
    *kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++*kernels;
        }
    }
  }
  // per-node priorities: the Hessian branch was captured from the high-priority stream
  e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return set_error(ELF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return ELF_OK;
}

// Single-iteration graphs for both buffer parities and, when tracing is off, graphs of kGraphIters
// iterations (an even count: they return to the parity they start from), which save the launch gaps
// between iterations on small problems.
int build_graph(elf_handle h) {
  for (int p = 0; p < 2; ++p) {
    if (!h->graph[p])
      if (int rc = capture_iterations(h, p, 1, &h->graph[p], &h->graph_kernels)) return rc;
    if (!h->tracing && !h->graph_r[p])
      if (int rc = capture_iterations(h, p, kGraphIters, &h->graph_r[p], nullptr)) return rc;
  }
  return ELF_OK;
}

void destroy_graphs(elf_handle h) {
  for (cudaGraphExec_t* set : {h->graph, h->graph_r})
    for (int p = 0; p < 2; ++p)
      if (set[p]) {
        cudaGraphExecDestroy(set[p]);
        set[p] = nullptr;
      }
}

// Makes buffer 0 of Psi and P current (before writing a new state into them).
void reset_current(elf_handle h) {
  h->cur = 0;
  h->psi = h->psi_buf[0];
  h->pupil = h->pupil_buf[0];
}

// Powers gamma^(t+1) and bias corrections 1/(1 - gamma^(t+1)) of Eq. 19 for the
// iteration after t.
int upload_bias(elf_handle h, int t, cudaStream_t s) {
  static thread_local double gp[2];
  static thread_local float bc[2];
  gp[0] = std::pow(h->opt.gamma1, (double)(t + 1));
  gp[1] = std::pow(h->opt.gamma2, (double)(t + 1));
  bc[0] = (float)(1.0 / (1.0 - gp[0]));
  bc[1] = (float)(1.0 / (1.0 - gp[1]));
  ELF_CK(cudaMemcpyAsync(h->gp, gp, sizeof(gp), cudaMemcpyHostToDevice, s));
  ELF_CK(cudaMemcpyAsync(h->bc + 2 * h->cur, bc, sizeof(bc), cudaMemcpyHostToDevice, s));
  return ELF_OK;
}

int check(elf_handle h) {
  if (!h) return set_error(ELF_EINVAL, "null handle");
  return ELF_OK;
}

int copy_out(elf_handle h, void* dst, const void* src, size_t bytes) {
  ELF_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->user));
  ELF_CK(cudaStreamSynchronize(h->user));
  return ELF_OK;
}

}  // namespace

extern "C" {

int elf_default_options(elf_options* o) {
  if (!o) return set_error(ELF_EINVAL, "null options");
  o->fidelity = 0;
  o->omega_iso = 1;
  o->learn_pupil = 1;
  o->pupil_filter = 1;
  o->alpha = -1.0;
  o->beta = -1.0;
  o->gamma1 = 0.9;
  o->gamma2 = 0.999;
  o->s0_psi = 1.0;
  o->s0_pupil = 1e-2;
  o->eta_opt = 1e-8;
  o->eta_h = 1e-12;
  o->tau_fid = 1e-6;
  o->tau_h = 1e-4;
  o->tile_dft = 0;
  o->g_exponent = 1.0;
  o->tile_path = 0;
  return ELF_OK;
}

void elf_destroy(elf_handle h) {
  if (!h) return;
  destroy_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  for (cudaEvent_t ev : h->ev_stage)
    if (ev) cudaEventDestroy(ev);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_tile) cudaEventDestroy(h->ev_tile);
  if (h->ev_cost) cudaEventDestroy(h->ev_cost);
  if (h->ev_pu) cudaEventDestroy(h->ev_pu);
  if (h->paux) cudaStreamDestroy(h->paux);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->aux) cudaStreamDestroy(h->aux);
  delete h;
}

static int create_impl(const elf_problem* p, const elf_options* o, void* stream, elf_handle h) {
  const int n = p->n_lowres, u = p->upsample, K = p->n_led;
  if (!(n == 16 || n == 32 || n == 64 || n == 128 || n == 256))
    return set_error(ELF_EINVAL, "n_lowres must be 16, 32, 64, 128 or 256");
  if (u < 1 || !is_pow2(u) || (long)n * u > 1024 || n * u < 32)
    return set_error(ELF_EINVAL, "upsample must be a power of two with 32 <= n*u <= 1024");
  if (K < 1 || K > 65536) return set_error(ELF_EINVAL, "n_led must be in [1, 65536]");
  if (!p->k_xy) return set_error(ELF_EINVAL, "k_xy is null");
  if (!(p->na > 0 && p->wavelength_um > 0 && p->pixel_um > 0) || !std::isfinite(p->na) ||
      !std::isfinite(p->wavelength_um) || !std::isfinite(p->pixel_um))
    return set_error(ELF_EINVAL, "na, wavelength_um and pixel_um must be finite and positive");
  if (o) {
    h->opt = *o;
  } else {
    elf_default_options(&h->opt);
  }
  const elf_options& op = h->opt;
  if (!(op.gamma1 >= 0 && op.gamma1 < 1 && op.gamma2 >= 0 && op.gamma2 < 1 && op.tau_fid >= 0 && op.tau_h >= 0 &&
        op.eta_opt >= 0 && op.eta_h >= 0 && op.s0_psi >= 0 && op.s0_pupil >= 0 && std::isfinite(op.alpha) &&
        std::isfinite(op.beta) && op.fidelity >= 0 && op.fidelity <= 3 && (op.tile_dft == 0 || op.tile_dft == 1) &&
        (op.fidelity != 2 || (std::isfinite(op.g_exponent) && op.g_exponent > 0 && op.g_exponent <= 8)) &&
        op.tile_path >= 0 && op.tile_path <= 2))
    return set_error(ELF_EINVAL, "invalid options");
  const int M = p->n_mux <= 0 ? 1 : p->n_mux;
  if (M > K || K % M != 0) return set_error(ELF_EINVAL, "n_led must be a positive multiple of n_mux");
  if (M > 1 && op.tile_dft) return set_error(ELF_EINVAL, "multiplexed images (n_mux > 1) need tile_dft = 0");
  if (op.tile_path == 2 && (M > 1 || op.tile_dft))
    return set_error(ELF_EINVAL, "tile_path = 2 needs n_mux = 1 and tile_dft = 0");
  h->split = tile_split_selected(n, M, op.tile_dft, op.tile_path);
  h->mux = M;
  h->n_img = K / M;
  h->n = n;
  h->u = u;
  h->N = n * u;
  h->K = K;
  const int N = h->N;
  h->dk = 1.0 / ((double)n * p->pixel_um);
  // LED offsets (reading A3) and crop windows
  h->origin_h.resize(K);
  double best = 1e300;
  for (int k = 0; k < K; ++k) {
    const double kx = p->k_xy[2 * k], ky = p->k_xy[2 * k + 1];
    if (!std::isfinite(kx) || !std::isfinite(ky)) return set_error(ELF_EINVAL, "non-finite k_xy");
    const double cy = round_half_away(ky / h->dk), cx = round_half_away(kx / h->dk);
    const double oy = cy + (N / 2 - n / 2), ox = cx + (N / 2 - n / 2);
    if (oy < 0 || ox < 0 || oy + n > N || ox + n > N)
      return set_error(ELF_EINVAL, "LED " + std::to_string(k) + ": crop window outside the spectrum");
    h->origin_h[k] = make_int2((int)oy, (int)ox);
    const double r2 = kx * kx + ky * ky;
    if (r2 < best) {
      best = r2;
      h->centre = k;
    }
  }
  // pupil support (reading A4), rows are contiguous runs of a disc
  h->pupil_cut = p->na / p->wavelength_um;
  const double cut = h->pupil_cut * h->pupil_cut;
  std::vector<int> xs(n, 0), cnt(n, 0), off(n, 0), sidx_map(n * n, -1), supy, supx;
  int S = 0, Blo = -1, Bhi = -1;
  for (int jy = 0; jy < n; ++jy) {
    off[jy] = S;
    for (int jx = 0; jx < n; ++jx) {
      const double a = jx - n / 2, b = jy - n / 2;
      const double rho2 = (a * a + b * b) * h->dk * h->dk;
      if (rho2 <= cut) {
        if (cnt[jy] == 0) xs[jy] = jx;
        if (jx != xs[jy] + cnt[jy]) return set_error(ELF_EINVAL, "support row is not contiguous");
        cnt[jy]++;
        sidx_map[jy * n + jx] = S++;
        supy.push_back(jy);
        supx.push_back(jx);
        h->sidx_h.push_back(jy * n + jx);
      }
    }
    if (cnt[jy] > 0) {
      if (Blo < 0) Blo = jy;
      if (Bhi >= 0 && Bhi != jy - 1) return set_error(ELF_EINVAL, "support rows are not contiguous");
      Bhi = jy;
    }
  }
  if (S == 0) return set_error(ELF_EINVAL, "empty pupil support (NA/wavelength smaller than one spectral pixel)");
  h->S = S;
  h->Blo = Blo;
  h->nb = Bhi - Blo + 1;
  if (h->opt.tile_dft && (n != kTcN || h->nb > kTcBand))
    return set_error(ELF_EINVAL, "tile_dft = 1 needs n_lowres = 128 and a support band of at most 64 rows");
  h->cs = tile_cluster_size(n);
  h->rowsA = (h->nb + h->cs - 1) / h->cs;
  h->Q = pupil_chunks(K, S);
  h->hblocks = hess_blocks(N);
  // gather lists (Eq. 9): for every spectrum row y and 64-pixel segment of it, the LEDs whose support
  // chord on that row crosses the segment, in ascending LED order, each as {LED, offset of the row
  // in the LED's compact G minus its first x, pupil index - x, first covered x | chord length << 16}
  const int seg = gather_seg(N);
  h->tiles_x = N / seg;
  std::vector<int> sptr((size_t)N * h->tiles_x + 1, 0);
  std::vector<int4> sent;
  {
    std::vector<std::vector<int4>> lists((size_t)N * h->tiles_x);
    for (int k = 0; k < K; ++k) {
      const int oy = h->origin_h[k].x, ox = h->origin_h[k].y;
      for (int jy = 0; jy < n; ++jy) {
        if (cnt[jy] == 0) continue;
        const int y = oy + jy, lo = ox + xs[jy], hi = lo + cnt[jy];  // covered x in [lo, hi)
        const int4 e = make_int4(k, off[jy] - lo, jy * n - ox, lo | (cnt[jy] << 16));
        for (int tx = lo / seg; tx <= (hi - 1) / seg; ++tx) lists[(size_t)y * h->tiles_x + tx].push_back(e);
      }
    }
    for (size_t i = 0; i < lists.size(); ++i) {
      sptr[i + 1] = sptr[i] + (int)lists[i].size();
      sent.insert(sent.end(), lists[i].begin(), lists[i].end());
    }
  }
  if (sent.empty()) sent.push_back(make_int4(0, 0, 0, 0));
  // Gaussian 3x3, sigma = 1 px, normalised (note under Algorithm 1)
  const double e = std::exp(-0.5), tot = 1.0 + 2.0 * e;
  h->gw0 = (float)(1.0 / tot);
  h->gw1 = (float)(e / tot);

  // streams and events
  h->user = static_cast<cudaStream_t>(stream);
  ELF_CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  // the Hessian branch gets the highest priority so that its short kernels are
  // scheduled ahead of the queued tile-kernel CTAs instead of after them
  int prio_low = 0, prio_high = 0;
  ELF_CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  ELF_CK(cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_high));
  ELF_CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  ELF_CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  ELF_CK(cudaEventCreateWithFlags(&h->ev_tile, cudaEventDisableTiming));
  ELF_CK(cudaEventCreateWithFlags(&h->ev_cost, cudaEventDisableTiming));
  ELF_CK(cudaEventCreateWithFlags(&h->ev_pu, cudaEventDisableTiming));
  ELF_CK(cudaStreamCreateWithPriority(&h->paux, cudaStreamNonBlocking, prio_high));  // short pupil kernels first
  for (cudaEvent_t& ev : h->ev_stage) ELF_CK(cudaEventCreate(&ev));

  // device memory
  int rc;
  const size_t A = (size_t)N * N, B = (size_t)n * n;
  if ((rc = upload(h, &h->origin, h->origin_h))) return rc;
  if ((rc = upload(h, &h->row_xs, xs))) return rc;
  if ((rc = upload(h, &h->row_cnt, cnt))) return rc;
  if ((rc = upload(h, &h->row_off, off))) return rc;
  if ((rc = upload(h, &h->sup_y, supy))) return rc;
  if ((rc = upload(h, &h->sup_x, supx))) return rc;
  if ((rc = upload(h, &h->sidx_map, sidx_map))) return rc;
  if ((rc = upload(h, &h->seg_ptr, sptr))) return rc;
  if ((rc = upload(h, &h->seg_ent, sent))) return rc;
  if ((rc = upload(h, &h->tw_n, twiddles(n)))) return rc;
  if ((rc = upload(h, &h->tw_N, twiddles(N)))) return rc;
  const size_t nI = (size_t)h->n_img * B;
  if ((rc = dalloc(h, &h->I, nI))) return rc;
  if (op.fidelity >= 1 && (rc = dalloc(h, &h->Ig, nI))) return rc;
  if (M > 1) {
    if ((rc = dalloc(h, &h->Imod, (size_t)K * B))) return rc;
    if ((rc = dalloc(h, &h->mux_r, nI))) return rc;
    if ((rc = dalloc(h, &h->mux_f, nI))) return rc;
    if ((rc = dalloc(h, &h->mux_cost, (size_t)h->n_img * mux_blocks_per_image(n)))) return rc;
  }
  if ((rc = dalloc(h, &h->psi_buf[0], A))) return rc;
  if ((rc = dalloc(h, &h->psi_buf[1], A))) return rc;
  if ((rc = dalloc(h, &h->mu_psi, A))) return rc;
  if ((rc = dalloc(h, &h->v_psi, A))) return rc;
  if ((rc = dalloc(h, &h->delta_psi, A))) return rc;
  if ((rc = dalloc(h, &h->pupil_buf[0], B))) return rc;
  if ((rc = dalloc(h, &h->pupil_buf[1], B))) return rc;
  reset_current(h);
  if ((rc = dalloc(h, &h->mu_p, B))) return rc;
  if ((rc = dalloc(h, &h->v_p, B))) return rc;
  if ((rc = dalloc(h, &h->delta_p, B))) return rc;
  if ((rc = dalloc(h, &h->G, (size_t)K * S))) return rc;
  if ((rc = dalloc(h, &h->ot, A))) return rc;
  if ((rc = dalloc(h, &h->q, A))) return rc;
  if (N >= 512 && (rc = dalloc(h, &h->fft_tmp, A))) return rc;
  if ((rc = dalloc(h, &h->small, B))) return rc;
  if ((rc = dalloc(h, &h->part, (size_t)h->Q * S))) return rc;
  if ((rc = dalloc(h, &h->pdone, (size_t)(S + 255) / 256))) return rc;
  ELF_CK(cudaMemset(h->pdone, 0, sizeof(int) * (size_t)((S + 255) / 256)));
  if ((rc = dalloc(h, &h->psi_eval, A))) return rc;
  if ((rc = dalloc(h, &h->pupil_eval, B))) return rc;
  if ((rc = dalloc(h, &h->g_psi, A))) return rc;
  if ((rc = dalloc(h, &h->g_p, B))) return rc;
  if ((rc = dalloc(h, &h->pupil_unit, B))) return rc;
  if ((rc = dalloc(h, &h->cost_fid, (size_t)K))) return rc;
  if ((rc = dalloc(h, &h->cost_ff, (size_t)K * h->cs * tile_warps(n)))) return rc;
  if ((rc = dalloc(h, &h->tc_err, 1))) return rc;
  ELF_CK(cudaMemset(h->tc_err, 0, sizeof(int)));
  if ((rc = dalloc(h, &h->cost_h, (size_t)2 * h->hblocks))) return rc;
  if ((rc = dalloc(h, &h->ring, (size_t)3 * kCostRing))) return rc;
  if ((rc = dalloc(h, &h->weights, 2))) return rc;
  if ((rc = dalloc(h, &h->alpha_part, (size_t)alpha_blocks(K, n)))) return rc;
  if ((rc = dalloc(h, &h->out4, 4))) return rc;
  if ((rc = dalloc(h, &h->t_dev, 1))) return rc;
  if ((rc = dalloc(h, &h->norm_part, (size_t)2 * gather_blocks(N)))) return rc;
  if ((rc = dalloc(h, &h->norm_ring, (size_t)2 * kCostRing))) return rc;
  if ((rc = dalloc(h, &h->norm_state, 3))) return rc;
  if ((rc = dalloc(h, &h->flag, 1))) return rc;
  if ((rc = dalloc(h, &h->bc, 4))) return rc;
  if ((rc = dalloc(h, &h->gp, 2))) return rc;
  if (h->opt.tile_dft) {
    const size_t Kz = (size_t)K;
    if ((rc = dalloc(h, &h->tc_iX, Kz * kTcImgX))) return rc;
    if ((rc = dalloc(h, &h->tc_iY, Kz * kTcImgY))) return rc;
    if ((rc = dalloc(h, &h->tc_iW, Kz * kTcImgW))) return rc;
    if ((rc = dalloc(h, &h->tc_iZ, Kz * kTcImgZ))) return rc;
    if ((rc = dalloc(h, &h->tc_Ot, Kz * kTcN * kTcN))) return rc;
    // rows 64..127 of the Z images are never written by the kernels and must read as zero
    ELF_CK(cudaMemset(h->tc_iZ, 0, Kz * kTcImgZ));
    // band DFT operands, FP64 on the host, split into BF16 hi + lo images
    for (int i = 0; i < 4; ++i)
      if ((rc = upload(h, &h->tc_c[i], tc_constant_image(i, h->Blo, h->nb)))) return rc;
    ELF_CK(prepare_tc());
  }
  ELF_CK(prepare_tile(n, h->rowsA));
  if (h->split) {
    if ((rc = dalloc(h, &h->band_in, (size_t)K * h->nb * n))) return rc;
    if ((rc = dalloc(h, &h->band_out, (size_t)K * h->nb * n))) return rc;
    ELF_CK(prepare_tile_split(n));
  }
  ELF_CK(prepare_fft(n));
  ELF_CK(prepare_fft(N));
  ELF_CK(launch_support_pupil(h->pupil_unit, h->sidx_map, n, h->user));
  ELF_CK(cudaMemsetAsync(h->t_dev, 0, sizeof(int), h->user));
  ELF_CK(cudaMemsetAsync(h->norm_state, 0, 3 * sizeof(int), h->user));
  ELF_CK(cudaMemsetAsync(h->norm_ring, 0, 2 * kCostRing * sizeof(double), h->user));
  ELF_CK(cudaMemsetAsync(h->ring, 0, 3 * kCostRing * sizeof(double), h->user));
  ELF_CK(cudaStreamSynchronize(h->user));
  return ELF_OK;
}

int elf_create(const elf_problem* p, const elf_options* o, void* stream, elf_handle* out) {
  if (!p || !out) return set_error(ELF_EINVAL, "null argument");
  *out = nullptr;
  elf_handle h = new elf_handle_s();
  const int rc = create_impl(p, o, stream, h);
  if (rc != ELF_OK) {
    elf_destroy(h);
    return rc;
  }
  *out = h;
  return ELF_OK;
}

}  // extern "C"

namespace elf {

// Initial state of elf_set_measurements from the measurements already in h->I,
// enqueued on the handle's stream without synchronising.
int init_state_async(elf_handle h) {
  const size_t B = (size_t)h->n * h->n, A = (size_t)h->N * h->N;
  cudaStream_t s = h->user;
  // alpha = beta (Eqs. 16-17) and the initial state (reading A9)
  if (h->opt.fidelity >= 1) {  // the measured side g(max(I, 0)), also what Eqs. 16-17 read
    ELF_CK(launch_gmap(h->I, h->Ig, (size_t)h->n_img * B, h->opt.fidelity, (float)h->opt.g_exponent, s));
    ELF_CK(launch_alpha(h->Ig, h->n_img, h->n, 0, h->alpha_part, h->weights, h->opt.alpha, h->opt.beta, s));
  } else {
    ELF_CK(launch_alpha(h->I, h->n_img, h->n, 0, h->alpha_part, h->weights, h->opt.alpha, h->opt.beta, s));
  }
  // Psi0 from the image that holds the centre LED (its own image when mux = 1)
  ELF_CK(launch_init_small(h->I + (size_t)(h->centre / h->mux) * B, h->small, h->n, s));
  ELF_CK(launch_fft2(h->small, h->n, false, h->tw_n, s));
  reset_current(h);  // the initial Psi goes into the first buffer
  ELF_CK(launch_embed(h->small, h->psi, h->n, h->N, h->origin_h[h->centre].x, h->origin_h[h->centre].y,
                      (float)(h->u * h->u), s));
  ELF_CK(launch_fill_f2(h->mu_psi, A, make_float2(0.f, 0.f), s));
  ELF_CK(launch_fill_f(h->v_psi, A, 0.f, s));
  ELF_CK(launch_fill_f(h->delta_psi, A, (float)(h->opt.s0_psi * h->opt.s0_psi), s));
  ELF_CK(launch_support_pupil(h->pupil, h->sidx_map, h->n, s));
  ELF_CK(launch_fill_f2(h->mu_p, B, make_float2(0.f, 0.f), s));
  ELF_CK(launch_fill_f(h->v_p, B, 0.f, s));
  ELF_CK(launch_fill_f(h->delta_p, B, (float)(h->opt.s0_pupil * h->opt.s0_pupil), s));
  ELF_CK(cudaMemsetAsync(h->t_dev, 0, sizeof(int), s));
  ELF_CK(cudaMemsetAsync(h->norm_state, 0, 3 * sizeof(int), s));
  ELF_CK(launch_init_bias(h->bc + 2 * h->cur, h->gp, h->opt.gamma1, h->opt.gamma2, s));
  h->have_meas = true;
  return ELF_OK;
}

// Asynchronous job pieces for the serving scheduler (server.cu).
int handle_set_measurements_async(elf_handle h, const float* I) {
  ELF_CK(cudaMemcpyAsync(h->I, I, (size_t)h->n_img * h->n * h->n * sizeof(float), cudaMemcpyDefault, h->user));
  return init_state_async(h);
}

int handle_get_object_async(elf_handle h, float* obj) {
  const size_t A = (size_t)h->N * h->N;
  ELF_CK(launch_fft2(h->ot, h->N, true, h->tw_N, h->user, h->psi, h->fft_tmp));  // reads Psi, writes ot
  ELF_CK(launch_sign_scale(h->ot, h->ot, h->N, (float)(1.0 / (double)A), h->user));
  ELF_CK(cudaMemcpyAsync(obj, h->ot, A * sizeof(float2), cudaMemcpyDefault, h->user));
  return ELF_OK;
}

size_t handle_device_bytes(elf_handle h) { return h->device_bytes; }
cudaStream_t handle_stream(elf_handle h) { return h->user; }
int handle_sizes(elf_handle h, int* n, int* N, int* K) {
  *n = h->n;
  *N = h->N;
  *K = h->K;
  return ELF_OK;
}
int handle_set_error(int code, const char* msg) { return set_error(code, msg); }
int handle_image_info(elf_handle h, int* n, int* N, int* n_img) {
  *n = h->n;
  *N = h->N;
  *n_img = h->n_img;
  return ELF_OK;
}
// Dark-field images (Eq. 21): every LED of the image has |c_n| dk > NA / lambda.
int handle_darkfield(elf_handle h, std::vector<unsigned char>& dark) {
  dark.assign(h->n_img, 1);
  const int off = h->N / 2 - h->n / 2;
  for (int k = 0; k < h->K; ++k) {
    const double cy = h->origin_h[k].x - off, cx = h->origin_h[k].y - off;
    if (std::sqrt(cy * cy + cx * cx) * h->dk <= h->pupil_cut) dark[k / h->mux] = 0;
  }
  return ELF_OK;
}

}  // namespace elf

extern "C" int elf_set_measurements(elf_handle h, const float* I, int is_device) {
  if (int rc = check(h)) return rc;
  if (!I) return set_error(ELF_EINVAL, "null measurements");
  (void)is_device;
  const size_t B = (size_t)h->n * h->n;
  cudaStream_t s = h->user;
  ELF_CK(cudaMemcpyAsync(h->I, I, (size_t)h->n_img * B * sizeof(float), cudaMemcpyDefault, s));
  ELF_CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
  ELF_CK(launch_count_nonfinite(h->I, (size_t)h->n_img * B, h->flag, s));
  int bad = 0;
  ELF_CK(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  ELF_CK(cudaStreamSynchronize(s));
  if (bad) {
    h->have_meas = false;
    return set_error(ELF_EINVAL, "measurements contain NaN or Inf");
  }
  if (int rc = init_state_async(h)) return rc;
  h->shard_open = false;
  ELF_CK(cudaStreamSynchronize(s));
  return ELF_OK;
}

extern "C" {

int elf_step(elf_handle h, int n_iter) {
  if (int rc = check(h)) return rc;
  if (!h->have_meas) return set_error(ELF_ESTATE, "elf_step before elf_set_measurements");
  if (h->shard_open) return set_error(ELF_ESTATE, "elf_step inside a sharded iteration (elf_shard_finish first)");
  if (n_iter < 0) return set_error(ELF_EINVAL, "negative n_iter");
  if (int rc = build_graph(h)) return rc;
  for (; !h->tracing && n_iter >= kGraphIters; n_iter -= kGraphIters)
    ELF_CK(cudaGraphLaunch(h->graph_r[h->cur], h->user));  // even count: the parity is unchanged
  for (int i = 0; i < n_iter; ++i) {
    ELF_CK(cudaGraphLaunch(h->graph[h->cur], h->user));
    h->cur ^= 1;  // the iteration's Psi^(t+1) and P^(t+1) are in the other buffers
    h->psi = h->psi_buf[h->cur];
    if (h->opt.learn_pupil) h->pupil = h->pupil_buf[h->cur];
  }
  return ELF_OK;
}

// ---- LED sharding: one iteration split around an exchange of the per-LED tile results
static int shard_check(elf_handle h, int k0, int k1) {
  if (int rc = check(h)) return rc;
  if (h->mux > 1 || h->opt.tile_dft) return set_error(ELF_EINVAL, "sharding needs n_mux = 1 and tile_dft = 0");
  if (k0 < 0 || k1 < k0 || k1 > h->K) return set_error(ELF_EINVAL, "LED range outside [0, n_led]");
  return ELF_OK;
}

int elf_shard_row_floats(elf_handle h) {
  if (int rc = check(h)) return rc;
  return 2 * (h->S + h->cs);
}

int elf_shard_tiles(elf_handle h, int led_begin, int led_end) {
  if (int rc = shard_check(h, led_begin, led_end)) return rc;
  if (!h->have_meas) return set_error(ELF_ESTATE, "elf_shard_tiles before elf_set_measurements");
  if (h->shard_open) return set_error(ELF_ESTATE, "elf_shard_tiles twice without elf_shard_finish");
  const int q = h->cur;
  const bool lp = h->opt.learn_pupil != 0;
  if (int rc = enqueue_iteration(h, 0, h->user, h->psi_buf[q], h->pupil_buf[lp ? q : 0], h->psi_buf[q ^ 1],
                                 lp ? h->pupil_buf[q ^ 1] : nullptr, kPartFront, led_begin, led_end))
    return rc;
  h->shard_open = true;
  h->shard_k0 = led_begin;
  h->shard_k1 = led_end;
  return ELF_OK;
}

int elf_shard_export(elf_handle h, int led_begin, int led_end, float* dst, int is_device) {
  if (int rc = shard_check(h, led_begin, led_end)) return rc;
  if (!dst) return set_error(ELF_EINVAL, "null destination");
  const size_t nl = (size_t)(led_end - led_begin), gb = nl * h->S * sizeof(float2);
  ELF_CK(cudaMemcpyAsync(dst, h->G + (size_t)led_begin * h->S, gb, cudaMemcpyDefault, h->user));
  ELF_CK(cudaMemcpyAsync(reinterpret_cast<char*>(dst) + gb, h->cost_ff + (size_t)led_begin * h->cs,
                         nl * h->cs * sizeof(float2), cudaMemcpyDefault, h->user));
  if (!is_device) ELF_CK(cudaStreamSynchronize(h->user));
  return ELF_OK;
}

int elf_shard_import(elf_handle h, int led_begin, int led_end, const float* src, int is_device) {
  if (int rc = shard_check(h, led_begin, led_end)) return rc;
  if (!src) return set_error(ELF_EINVAL, "null source");
  (void)is_device;
  const size_t nl = (size_t)(led_end - led_begin), gb = nl * h->S * sizeof(float2);
  ELF_CK(cudaMemcpyAsync(h->G + (size_t)led_begin * h->S, src, gb, cudaMemcpyDefault, h->user));
  ELF_CK(cudaMemcpyAsync(h->cost_ff + (size_t)led_begin * h->cs, reinterpret_cast<const char*>(src) + gb,
                         nl * h->cs * sizeof(float2), cudaMemcpyDefault, h->user));
  return ELF_OK;
}

int elf_shard_finish(elf_handle h) {
  if (int rc = check(h)) return rc;
  if (!h->shard_open) return set_error(ELF_ESTATE, "elf_shard_finish without elf_shard_tiles");
  const int q = h->cur;
  const bool lp = h->opt.learn_pupil != 0;
  h->shard_open = false;
  if (int rc = enqueue_iteration(h, 0, h->user, h->psi_buf[q], h->pupil_buf[lp ? q : 0], h->psi_buf[q ^ 1],
                                 lp ? h->pupil_buf[q ^ 1] : nullptr, kPartBack))
    return rc;
  h->cur ^= 1;  // Psi^(t+1) and P^(t+1) are in the other buffers, as after elf_step
  h->psi = h->psi_buf[h->cur];
  if (lp) h->pupil = h->pupil_buf[h->cur];
  return ELF_OK;
}

int elf_get_spectrum(elf_handle h, float* psi, int is_device) {
  if (int rc = check(h)) return rc;
  if (!psi) return set_error(ELF_EINVAL, "null output");
  (void)is_device;
  return copy_out(h, psi, h->psi, (size_t)h->N * h->N * sizeof(float2));
}

int elf_get_pupil(elf_handle h, float* pupil, int is_device) {
  if (int rc = check(h)) return rc;
  if (!pupil) return set_error(ELF_EINVAL, "null output");
  (void)is_device;
  return copy_out(h, pupil, h->pupil, (size_t)h->n * h->n * sizeof(float2));
}

int elf_get_object(elf_handle h, float* obj, int is_device) {
  if (int rc = check(h)) return rc;
  if (!obj) return set_error(ELF_EINVAL, "null output");
  (void)is_device;
  const size_t A = (size_t)h->N * h->N;
  ELF_CK(launch_fft2(h->ot, h->N, true, h->tw_N, h->user, h->psi, h->fft_tmp));  // reads Psi, writes ot
  ELF_CK(launch_sign_scale(h->ot, h->ot, h->N, (float)(1.0 / (double)A), h->user));
  return copy_out(h, obj, h->ot, A * sizeof(float2));
}

int elf_get_costs(elf_handle h, double* out, int max_iter) {
  if (int rc = check(h)) return rc;
  if (!out || max_iter < 0) return set_error(ELF_EINVAL, "bad output");
  int t = 0;
  ELF_CK(cudaMemcpyAsync(&t, h->t_dev, sizeof(int), cudaMemcpyDeviceToHost, h->user));
  ELF_CK(cudaStreamSynchronize(h->user));
  if (h->tc_err) {
    int bad = 0;
    ELF_CK(cudaMemcpy(&bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return set_error(ELF_ETIMEOUT, "a bounded device wait ran out; results are invalid");
  }
  int count = t < max_iter ? t : max_iter;
  if (count > kCostRing) count = kCostRing;
  std::vector<double> ring(3 * kCostRing);
  ELF_CK(cudaMemcpy(ring.data(), h->ring, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < count; ++i) {
    const int it = t - count + i;
    std::memcpy(out + 3 * i, ring.data() + 3 * (it % kCostRing), 3 * sizeof(double));
  }
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < 3; ++j)
      if (!std::isfinite(out[3 * i + j])) return set_error(ELF_ENUMERIC, "non-finite cost");
  return count;
}

int elf_selftest_wait_timeout(elf_handle h, long long limit, double* ms) {
  if (int rc = check(h)) return rc;
  if (limit < 1 || limit > (1LL << 30)) return set_error(ELF_EINVAL, "limit must be in [1, 2^30]");
  cudaEvent_t a = nullptr, b = nullptr;
  ELF_CK(cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, h->user);
  if (e == cudaSuccess) e = launch_wait_timeout(h->tc_err, limit, h->user);
  if (e == cudaSuccess) e = cudaEventRecord(b, h->user);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return set_error(ELF_ECUDA, cudaGetErrorString(e));
  if (ms) *ms = t;
  return ELF_OK;
}

int elf_get_norms(elf_handle h, double* out, int max_iter) {
  if (int rc = check(h)) return rc;
  if (!out || max_iter < 0) return set_error(ELF_EINVAL, "bad output");
  // the most recent update's norms, if no later cost reduction has added them up yet
  const int nblk = gather_blocks(h->N);
  for (int p = 0; p < 2; ++p)
    ELF_CK(launch_norms_finalize(NormArgs{h->norm_part + (size_t)p * nblk, nblk, h->norm_state + p, h->norm_state + 2,
                                          h->norm_ring},
                                 h->user));
  int ns[3] = {0, 0, 0};
  ELF_CK(cudaMemcpyAsync(ns, h->norm_state, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->user));
  ELF_CK(cudaStreamSynchronize(h->user));
  const int t = ns[2];
  int count = t < max_iter ? t : max_iter;
  if (count > kCostRing) count = kCostRing;
  std::vector<double> ring(2 * kCostRing);
  ELF_CK(cudaMemcpy(ring.data(), h->norm_ring, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < count; ++i) {
    const int it = t - count + i;
    std::memcpy(out + 2 * i, ring.data() + 2 * (it % kCostRing), 2 * sizeof(double));
  }
  for (int i = 0; i < 2 * count; ++i)
    if (!std::isfinite(out[i])) return set_error(ELF_ENUMERIC, "non-finite norm");
  return count;
}

int elf_get_state(elf_handle h, const elf_state* st, int is_device) {
  if (int rc = check(h)) return rc;
  if (!st) return set_error(ELF_EINVAL, "null state");
  (void)is_device;
  const size_t A = (size_t)h->N * h->N, B = (size_t)h->n * h->n;
  cudaStream_t s = h->user;
  struct {
    void* dst;
    const void* src;
    size_t bytes;
  } cp[] = {{st->psi, h->psi, A * 8},       {st->mu_psi, h->mu_psi, A * 8},    {st->v_psi, h->v_psi, A * 4},
            {st->delta_psi, h->delta_psi, A * 4}, {st->pupil, h->pupil, B * 8}, {st->mu_pupil, h->mu_p, B * 8},
            {st->v_pupil, h->v_p, B * 4},   {st->delta_pupil, h->delta_p, B * 4}};
  for (auto& c : cp)
    if (c.dst) ELF_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDefault, s));
  int t = 0;
  double w[2] = {0, 0};
  ELF_CK(cudaMemcpyAsync(&t, h->t_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  ELF_CK(cudaMemcpyAsync(w, h->weights, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ELF_CK(cudaStreamSynchronize(s));
  elf_state* mst = const_cast<elf_state*>(st);
  mst->t = t;
  mst->alpha = w[0];
  mst->beta = w[1];
  return ELF_OK;
}

int elf_set_state(elf_handle h, const elf_state* st, int is_device) {
  if (int rc = check(h)) return rc;
  if (!st || !st->psi || !st->mu_psi || !st->v_psi || !st->delta_psi || !st->pupil || !st->mu_pupil ||
      !st->v_pupil || !st->delta_pupil)
    return set_error(ELF_EINVAL, "incomplete state");
  if (st->t < 0 || !std::isfinite(st->alpha) || !std::isfinite(st->beta) || st->alpha < 0 || st->beta < 0)
    return set_error(ELF_EINVAL, "invalid t, alpha or beta");
  if (!h->have_meas) return set_error(ELF_ESTATE, "elf_set_state before elf_set_measurements");
  if (h->shard_open) return set_error(ELF_ESTATE, "elf_set_state inside a sharded iteration");
  (void)is_device;
  const size_t A = (size_t)h->N * h->N, B = (size_t)h->n * h->n;
  cudaStream_t s = h->user;
  ELF_CK(cudaMemcpyAsync(h->psi, st->psi, A * 8, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->mu_psi, st->mu_psi, A * 8, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->v_psi, st->v_psi, A * 4, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->delta_psi, st->delta_psi, A * 4, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->pupil, st->pupil, B * 8, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->mu_p, st->mu_pupil, B * 8, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->v_p, st->v_pupil, B * 4, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->delta_p, st->delta_pupil, B * 4, cudaMemcpyDefault, s));
  const int t = st->t;
  const double w[2] = {st->alpha, st->beta};
  ELF_CK(cudaMemcpyAsync(h->t_dev, &t, sizeof(int), cudaMemcpyHostToDevice, s));
  const int ns[3] = {0, 0, t};  // nothing pending; the norm ring continues at the state's iteration count
  ELF_CK(cudaMemcpyAsync(h->norm_state, ns, 3 * sizeof(int), cudaMemcpyHostToDevice, s));
  ELF_CK(cudaMemcpyAsync(h->weights, w, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  if (int rc = upload_bias(h, t, s)) return rc;
  ELF_CK(cudaStreamSynchronize(s));
  return ELF_OK;
}

int elf_cost_grad(elf_handle h, const float* psi, const float* pupil, double* costs4, float* g_psi, float* g_pupil,
                  int is_device) {
  if (int rc = check(h)) return rc;
  if (!psi || !pupil) return set_error(ELF_EINVAL, "null psi or pupil");
  if (!h->have_meas) return set_error(ELF_ESTATE, "elf_cost_grad before elf_set_measurements");
  if (h->shard_open) return set_error(ELF_ESTATE, "elf_cost_grad inside a sharded iteration");
  (void)is_device;
  const size_t A = (size_t)h->N * h->N, B = (size_t)h->n * h->n;
  cudaStream_t s = h->user;
  ELF_CK(cudaMemcpyAsync(h->psi_eval, psi, A * 8, cudaMemcpyDefault, s));
  ELF_CK(cudaMemcpyAsync(h->pupil_eval, pupil, B * 8, cudaMemcpyDefault, s));
  if (int rc = enqueue_iteration(h, 1, s, h->psi_eval, h->pupil_eval, nullptr, nullptr)) return rc;
  if (g_psi) ELF_CK(cudaMemcpyAsync(g_psi, h->g_psi, A * 8, cudaMemcpyDefault, s));
  if (g_pupil) ELF_CK(cudaMemcpyAsync(g_pupil, h->g_p, B * 8, cudaMemcpyDefault, s));
  double c[4];
  ELF_CK(cudaMemcpyAsync(c, h->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ELF_CK(cudaStreamSynchronize(s));
  if (h->tc_err) {
    int bad = 0;
    ELF_CK(cudaMemcpy(&bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return set_error(ELF_ETIMEOUT, "a bounded device wait ran out; results are invalid");
  }
  if (costs4) std::memcpy(costs4, c, sizeof(c));
  for (double v : c)
    if (!std::isfinite(v)) return set_error(ELF_ENUMERIC, "non-finite cost");
  return ELF_OK;
}

int elf_simulate(elf_handle h, const float* obj, float* I_out, int is_device) {
  if (int rc = check(h)) return rc;
  if (!obj || !I_out) return set_error(ELF_EINVAL, "null argument");
  const size_t A = (size_t)h->N * h->N, B = (size_t)h->n * h->n;
  cudaStream_t s = h->user;
  // Psi = fftshift(DFT_N(O)) = DFT_N((-1)^(x+y) O)
  ELF_CK(cudaMemcpyAsync(h->psi_eval, obj, A * 8, cudaMemcpyDefault, s));
  ELF_CK(launch_sign_scale(h->psi_eval, h->psi_eval, h->N, 1.f, s));
  ELF_CK(launch_fft2(h->psi_eval, h->N, false, h->tw_N, s, nullptr, h->fft_tmp));
  const size_t nI = (size_t)h->n_img * B;  // K/M images of Eq. 1
  float* dst = I_out;
  float* staging = nullptr;
  if (!is_device) {
    ELF_CK(cudaMalloc(&staging, nI * sizeof(float)));
    dst = staging;
  }
  TileArgs ta{};
  ta.psi = h->psi_eval;
  ta.pupil = h->pupil_unit;
  ta.origin = h->origin;
  ta.row_xs = h->row_xs;
  ta.row_cnt = h->row_cnt;
  ta.row_off = h->row_off;
  ta.tw = h->tw_n;
  ta.I_out = h->mux > 1 ? h->Imod : dst;  // per-LED |o|^2, summed per image below when M > 1
  ta.cost_ff = h->cost_ff;
  ta.err = h->tc_err;
  ta.N = h->N;
  ta.K = h->K;
  ta.S = h->S;
  ta.Blo = h->Blo;
  ta.nb = h->nb;
  ta.rowsA = h->rowsA;
  ta.scale = (float)(1.0 / ((double)h->u * h->u * (double)h->n * h->n));
  ta.mode = 1;
  ta.mux = h->mux;
  cudaError_t e = launch_tile(ta, h->n, s);
  if (e == cudaSuccess && h->mux > 1) e = launch_mux_sum(h->Imod, dst, h->n_img, h->mux, h->n, s);
  if (e == cudaSuccess && staging) e = cudaMemcpyAsync(I_out, staging, nI * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (staging) cudaFree(staging);
  if (e != cudaSuccess) return set_error(ELF_ECUDA, std::string("elf_simulate: ") + cudaGetErrorString(e));
  int bad = 0;
  ELF_CK(cudaMemcpy(&bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) return set_error(ELF_ETIMEOUT, "a bounded device wait ran out; results are invalid");
  return ELF_OK;
}

int elf_get_tile_grads(elf_handle h, float* G_out, int is_device) {
  if (int rc = check(h)) return rc;
  if (!G_out) return set_error(ELF_EINVAL, "null output");
  (void)is_device;
  return copy_out(h, G_out, h->G, (size_t)h->K * h->S * sizeof(float2));
}

int elf_get_support(elf_handle h, int* idx) {
  if (int rc = check(h)) return rc;
  if (idx) std::memcpy(idx, h->sidx_h.data(), h->sidx_h.size() * sizeof(int));
  return h->S;
}

int elf_get_weights(elf_handle h, double* alpha, double* beta) {
  if (int rc = check(h)) return rc;
  double w[2];
  ELF_CK(cudaMemcpyAsync(w, h->weights, sizeof(w), cudaMemcpyDeviceToHost, h->user));
  ELF_CK(cudaStreamSynchronize(h->user));
  if (alpha) *alpha = w[0];
  if (beta) *beta = w[1];
  return ELF_OK;
}

int elf_set_tracing(elf_handle h, int enable) {
  if (int rc = check(h)) return rc;
  const bool en = enable != 0;
  if (en != h->tracing) {
    ELF_CK(cudaStreamSynchronize(h->user));
    destroy_graphs(h);
  }
  h->tracing = en;
  return ELF_OK;
}

int elf_get_stage_times(elf_handle h, float* ms, int max_stages) {
  if (int rc = check(h)) return rc;
  if (!ms || max_stages < 0) return set_error(ELF_EINVAL, "bad output");
  if (!h->tracing) return set_error(ELF_ESTATE, "tracing is off");
  ELF_CK(cudaStreamSynchronize(h->user));
  const int n = max_stages < ELF_NSTAGES ? max_stages : ELF_NSTAGES;
  for (int i = 0; i < n; ++i) {
    float t = -1.f;
    if (cudaEventElapsedTime(&t, h->ev_stage[2 * i], h->ev_stage[2 * i + 1]) != cudaSuccess) t = -1.f;
    ms[i] = t;
  }
  cudaGetLastError();  // stages that never ran leave a benign "not ready" error behind
  return n;
}

int elf_get_stage_spans(elf_handle h, float* spans, int max_stages) {
  if (int rc = check(h)) return rc;
  if (!spans || max_stages < 0) return set_error(ELF_EINVAL, "bad output");
  if (!h->tracing) return set_error(ELF_ESTATE, "tracing is off");
  ELF_CK(cudaStreamSynchronize(h->user));
  const int n = max_stages < ELF_NSTAGES ? max_stages : ELF_NSTAGES;
  for (int i = 0; i < 2 * n; ++i) {
    float t = -1.f;
    if (cudaEventElapsedTime(&t, h->ev_stage[0], h->ev_stage[i]) != cudaSuccess) t = -1.f;
    spans[i] = t;
  }
  cudaGetLastError();  // stages that never ran leave a benign "not ready" error behind
  return n;
}

int elf_graph_kernel_count(elf_handle h) {
  if (int rc = check(h)) return rc;
  if (int rc = build_graph(h)) return rc;
  return h->graph_kernels;
}

const char* elf_strerror(int code) {
  switch (code) {
    case ELF_OK: return "ok";
    case ELF_EINVAL: return "invalid argument";
    case ELF_ENOMEM: return "out of device memory";
    case ELF_ECUDA: return "CUDA error";
    case ELF_ENUMERIC: return "non-finite cost";
    case ELF_ETIMEOUT: return "timeout";
    case ELF_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* elf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
