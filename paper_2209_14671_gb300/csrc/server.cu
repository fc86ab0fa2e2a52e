// Continuous-batching server for many independent Elfpie reconstructions.
//
// Requests (a problem, its measurements, an iteration count) queue on the host.
// elf_server_progress admits queued requests in arrival order while the device
// memory budget and the slot count allow, and retires finished ones without
// blocking.  An admitted request gets a handle from a pool keyed by its problem
// and options (handles are created once and reused, so admission allocates only
// the first time a shape is seen), and its whole job is enqueued at once on that
// handle's own stream: the copy of its measurements and the initial state
// (elf_set_measurements without synchronisation), its elf_step iterations (the
// iteration graph), the object transform and its copy into a pooled pinned
// result buffer, and a completion event.  Jobs of different requests therefore
// overlap on the device; each job's arithmetic is exactly that of a lone run, so
// results do not depend on what else is in flight.  When admission needs room,
// idle pooled handles are destroyed, least recently used first.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <string>
#include <vector>

#include "../../include/elfpie.h"
#include "internal.cuh"

namespace elf {
int handle_set_measurements_async(elf_handle h, const float* I);
int handle_get_object_async(elf_handle h, float* obj);
size_t handle_device_bytes(elf_handle h);
cudaStream_t handle_stream(elf_handle h);
int handle_set_error(int code, const char* msg);
}  // namespace elf

namespace {

struct Request {
  long long tag = 0;
  std::string key;
  elf_problem prob{};
  std::vector<float> k_xy;
  elf_options opt{};
  const float* I = nullptr;  // caller's buffer, valid until the result is collected
  int n_iter = 0;
  int N = 0;
  elf_handle h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* result = nullptr;   // pinned N x N complex
};

struct Pooled {
  elf_handle h = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  unsigned long long last_use = 0;
};

std::string make_key(const elf_problem& p, const elf_options& o) {
  std::string k;
  auto put = [&](const void* d, size_t n) { k.append(static_cast<const char*>(d), n); };
  put(&p.n_lowres, sizeof(int));
  put(&p.upsample, sizeof(int));
  put(&p.n_led, sizeof(int));
  const int mux = p.n_mux <= 0 ? 1 : p.n_mux;
  put(&mux, sizeof(int));
  put(&p.na, sizeof(double));
  put(&p.wavelength_um, sizeof(double));
  put(&p.pixel_um, sizeof(double));
  put(p.k_xy, sizeof(float) * 2 * (size_t)p.n_led);
  put(&o, sizeof(o));
  return k;
}

// Device bytes a handle of this problem will hold (the allocations of elf_create).
size_t estimate_bytes(const elf_problem& p, int tile_dft, int fidelity, int tile_path) {
  const size_t n = p.n_lowres, N = (size_t)p.n_lowres * p.upsample, K = p.n_led;
  const size_t M = p.n_mux <= 0 ? 1 : p.n_mux, nI = K / M;  // measured images
  const size_t A = N * N, B = n * n, S = B;  // the support is at most the whole pupil grid
  // Psi-sized: 8 complex (Psi double-buffered, the transforms' scratch) + 2 real; per LED: I and G plus the Eq. 18 partials and the tile kernel's
  // per-warp cost pairs; pupil-sized: 8 complex + 3 real/int; 1 MB for the remaining tables,
  // twiddles and reductions
  const size_t cost_pairs = 8 * (size_t)elf::tile_cluster_size((int)n) * (size_t)elf::tile_warps((int)n);
  // the tensor-core tile path adds its per-LED operand images and O', and 640 KB of constants
  const size_t tc = tile_dft ? K * (elf::kTcImgX + elf::kTcImgY + elf::kTcImgW + elf::kTcImgZ +
                                    8 * (size_t)elf::kTcN * elf::kTcN) + (640u << 10)
                             : 0;
  // the amplitude fidelity and the Sec. 6.3 maps keep a mapped copy of the measurements
  const size_t gmap = fidelity >= 1 ? 4 * nI * B : 0;
  // multiplexed images: per-LED |o|^2, per-image residual and factor, per-block cost partials
  const size_t mux = M > 1 ? 4 * K * B + 8 * nI * B + 8 * nI * (size_t)elf::mux_blocks_per_image((int)n) : 0;
  // the split tile path keeps two support bands per LED (at most n rows of n complex each)
  const size_t split = elf::tile_split_selected((int)n, (int)M, tile_dft, tile_path) ? 16 * K * B : 0;
  return 8 * A * 8 + 4 * A * 2 + 4 * nI * B + 16 * K * S + cost_pairs * K + 8 * B * 8 + 4 * B * 3 + tc + gmap +
         mux + split + (1u << 20);
}

}  // namespace

struct elf_server_s {
  size_t budget = 0, used = 0;
  int max_active = 0;
  unsigned long long clock = 0;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<long long, Request*> finished;
  std::multimap<std::string, Pooled> idle;
  std::map<int, std::vector<float*>> pinned_free;  // result buffers by N
  int n_admitted = 0, n_created = 0;
};

namespace {

int fail(int code, const std::string& msg) { return elf::handle_set_error(code, msg.c_str()); }

float* take_pinned(elf_server s, int N) {
  auto& v = s->pinned_free[N];
  if (!v.empty()) {
    float* p = v.back();
    v.pop_back();
    return p;
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, (size_t)N * N * 2 * sizeof(float)) != cudaSuccess) return nullptr;
  return static_cast<float*>(p);
}

void destroy_pooled(elf_server s, Pooled& p) {
  elf_destroy(p.h);
  if (p.stream) cudaStreamDestroy(p.stream);
  s->used -= p.bytes;
}

// Frees idle handles (least recently used first) until `need` more bytes fit.
bool make_room(elf_server s, size_t need) {
  while (s->used + need > s->budget && !s->idle.empty()) {
    auto victim = s->idle.begin();
    for (auto it = s->idle.begin(); it != s->idle.end(); ++it)
      if (it->second.last_use < victim->second.last_use) victim = it;
    destroy_pooled(s, victim->second);
    s->idle.erase(victim);
  }
  return s->used + need <= s->budget;
}

// Admits the request at the head of the queue if it fits; returns 1 if admitted,
// 0 if it must wait, < 0 on error.
int admit_one(elf_server s) {
  Request* r = s->queue.front();
  Pooled p;
  auto it = s->idle.find(r->key);
  if (it != s->idle.end()) {
    p = it->second;
    s->idle.erase(it);
  } else {
    const size_t est = estimate_bytes(r->prob, r->opt.tile_dft, r->opt.fidelity, r->opt.tile_path);
    if (!make_room(s, est)) return 0;
    if (cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ELF_ECUDA, "cudaStreamCreate failed");
    const int rc = elf_create(&r->prob, &r->opt, p.stream, &p.h);
    if (rc != ELF_OK) {
      cudaStreamDestroy(p.stream);
      return rc;
    }
    p.bytes = elf::handle_device_bytes(p.h);
    s->used += p.bytes;
    s->n_created++;
  }
  r->h = p.h;
  r->stream = p.stream;
  r->result = take_pinned(s, r->N);
  if (!r->result) return fail(ELF_ENOMEM, "pinned result buffer");
  if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess)
    return fail(ELF_ECUDA, "cudaEventCreate failed");
  int rc = elf::handle_set_measurements_async(r->h, r->I);
  if (rc == ELF_OK) rc = elf_step(r->h, r->n_iter);
  if (rc == ELF_OK) rc = elf::handle_get_object_async(r->h, r->result);
  if (rc != ELF_OK) return rc;
  if (cudaEventRecord(r->done, r->stream) != cudaSuccess) return fail(ELF_ECUDA, "cudaEventRecord failed");
  // keep the handle's bookkeeping in the request until it is retired
  s->queue.pop_front();
  s->active.push_back(r);
  s->n_admitted++;
  (void)p.last_use;
  return 1;
}

}  // namespace

extern "C" {

int elf_server_create(size_t budget_bytes, int max_active, elf_server* out) {
  if (!out || max_active < 1 || budget_bytes == 0) return fail(ELF_EINVAL, "bad server arguments");
  elf_server s = new elf_server_s();
  s->budget = budget_bytes;
  s->max_active = max_active;
  *out = s;
  return ELF_OK;
}

int elf_server_submit(elf_server s, const elf_problem* prob, const elf_options* opt, const float* I, int n_iter,
                      long long tag) {
  if (!s || !prob || !I || n_iter < 0) return fail(ELF_EINVAL, "bad submit arguments");
  if (!prob->k_xy || prob->n_led < 1) return fail(ELF_EINVAL, "bad problem");
  if (s->finished.count(tag)) return fail(ELF_EINVAL, "tag already in use");
  for (Request* q : s->queue)
    if (q->tag == tag) return fail(ELF_EINVAL, "tag already in use");
  for (Request* q : s->active)
    if (q->tag == tag) return fail(ELF_EINVAL, "tag already in use");
  if (estimate_bytes(*prob, opt ? opt->tile_dft : 0, opt ? opt->fidelity : 0, opt ? opt->tile_path : 0) > s->budget)
    return fail(ELF_ENOMEM, "request larger than the memory budget");
  Request* r = new Request();
  r->tag = tag;
  r->prob = *prob;
  r->k_xy.assign(prob->k_xy, prob->k_xy + 2 * (size_t)prob->n_led);
  r->prob.k_xy = r->k_xy.data();
  if (opt) {
    r->opt = *opt;
  } else {
    elf_default_options(&r->opt);
  }
  r->I = I;
  r->n_iter = n_iter;
  r->N = prob->n_lowres * prob->upsample;
  r->key = make_key(r->prob, r->opt);
  s->queue.push_back(r);
  return ELF_OK;
}

int elf_server_progress(elf_server s, long long* done_tags, int max_done, int* n_done) {
  if (!s || !n_done || (max_done > 0 && !done_tags)) return fail(ELF_EINVAL, "bad progress arguments");
  *n_done = 0;
  // retire finished jobs first so that their memory can be reused
  for (size_t i = 0; i < s->active.size();) {
    Request* r = s->active[i];
    const cudaError_t e = cudaEventQuery(r->done);
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (e != cudaSuccess) return fail(ELF_ECUDA, std::string("request failed: ") + cudaGetErrorString(e));
    Pooled p;
    p.h = r->h;
    p.stream = r->stream;
    p.bytes = elf::handle_device_bytes(r->h);
    p.last_use = ++s->clock;
    s->idle.emplace(r->key, p);
    r->h = nullptr;
    s->finished[r->tag] = r;
    s->active.erase(s->active.begin() + (long)i);
    if (*n_done < max_done) done_tags[(*n_done)++] = r->tag;
  }
  while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
    const int rc = admit_one(s);
    if (rc < 0) return rc;
    if (rc == 0) break;
  }
  return ELF_OK;
}

int elf_server_result(elf_server s, long long tag, float* obj) {
  if (!s || !obj) return fail(ELF_EINVAL, "bad result arguments");
  auto it = s->finished.find(tag);
  if (it == s->finished.end()) return fail(ELF_ESTATE, "request not finished (or unknown tag)");
  Request* r = it->second;
  std::memcpy(obj, r->result, (size_t)r->N * r->N * 2 * sizeof(float));
  s->pinned_free[r->N].push_back(r->result);
  cudaEventDestroy(r->done);
  s->finished.erase(it);
  delete r;
  return ELF_OK;
}

int elf_server_cancel(elf_server s, long long tag) {
  if (!s) return fail(ELF_EINVAL, "null server");
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if ((*it)->tag != tag) continue;
    delete *it;
    s->queue.erase(it);
    return ELF_OK;
  }
  for (size_t i = 0; i < s->active.size(); ++i) {
    Request* r = s->active[i];
    if (r->tag != tag) continue;
    // its whole job is on the device already: wait for it, keep the handle, drop the result
    const cudaError_t e = cudaEventSynchronize(r->done);
    if (e != cudaSuccess) return fail(ELF_ECUDA, std::string("request failed: ") + cudaGetErrorString(e));
    Pooled p;
    p.h = r->h;
    p.stream = r->stream;
    p.bytes = elf::handle_device_bytes(r->h);
    p.last_use = ++s->clock;
    s->idle.emplace(r->key, p);
    s->pinned_free[r->N].push_back(r->result);
    cudaEventDestroy(r->done);
    s->active.erase(s->active.begin() + (long)i);
    delete r;
    return ELF_OK;
  }
  auto it = s->finished.find(tag);
  if (it == s->finished.end()) return fail(ELF_EINVAL, "unknown tag");
  Request* r = it->second;
  s->pinned_free[r->N].push_back(r->result);
  cudaEventDestroy(r->done);
  s->finished.erase(it);
  delete r;
  return ELF_OK;
}

int elf_server_stats(elf_server s, size_t* used_bytes, int* n_active, int* n_queued, int* n_created) {
  if (!s) return fail(ELF_EINVAL, "null server");
  if (used_bytes) *used_bytes = s->used;
  if (n_active) *n_active = (int)s->active.size();
  if (n_queued) *n_queued = (int)s->queue.size();
  if (n_created) *n_created = s->n_created;
  return ELF_OK;
}

void elf_server_destroy(elf_server s) {
  if (!s) return;
  for (Request* r : s->active) cudaEventSynchronize(r->done);
  for (Request* r : s->active) {
    Pooled p;
    p.h = r->h;
    p.stream = r->stream;
    p.bytes = elf::handle_device_bytes(r->h);
    destroy_pooled(s, p);
    cudaEventDestroy(r->done);
    if (r->result) cudaFreeHost(r->result);
    delete r;
  }
  for (auto& kv : s->idle) destroy_pooled(s, kv.second);
  for (auto& kv : s->finished) {
    cudaEventDestroy(kv.second->done);
    cudaFreeHost(kv.second->result);
    delete kv.second;
  }
  for (Request* r : s->queue) delete r;
  for (auto& kv : s->pinned_free)
    for (float* p : kv.second) cudaFreeHost(p);
  delete s;
}

}  // extern "C"
