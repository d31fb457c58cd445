// C ABI of the tomo library: grid handle, multigrid hierarchy, preconditioned CG driver and
// the exact-gradient evaluation (Algorithm 1, exact branch; Eq. 4-5, Section III-D).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "host.h"

using namespace tomo;

namespace tomo {
thread_local std::string g_create_err;
thread_local std::string* g_cur_err = nullptr;

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e),
           what, file, line);
  if (g_cur_err) *g_cur_err = buf;
  return TOMO_ECUDA;
}
}  // namespace tomo

namespace {

tomo_status fail(tomo_grid* G, tomo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (G) G->err = buf;
  else g_create_err = buf;
  return st;
}

#define CK(...)                                                        \
  do {                                                                 \
    cudaError_t _e = (__VA_ARGS__);                                    \
    if (_e != cudaSuccess) {                                           \
      return fail(G, _e == cudaErrorMemoryAllocation ? TOMO_ENOMEM : TOMO_ECUDA, \
                  "CUDA error %d (%s) in %s (%s:%d)", (int)_e,         \
                  cudaGetErrorString(_e), #__VA_ARGS__, __FILE__, __LINE__); \
    }                                                                  \
  } while (0)

#define TRY(...)                           \
  do {                                     \
    tomo_status _s = (__VA_ARGS__);        \
    if (_s != TOMO_OK) return _s;          \
  } while (0)

template <typename T>
ElemConst<T> elem_const(const tomo_grid* G) {
  ElemConst<T> c;
  for (int k = 0; k < 8; ++k)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) c.blk[k][a][b] = (T)G->blk[k][a][b];
  c.k0diag = (T)G->k0diag;
  return c;
}

template <typename T>
DenseK0<T> dense_k0(const tomo_grid* G) {
  DenseK0<T> d;
  for (int q = 0; q < 576; ++q) d.k[q] = (T)G->K0[q];
  return d;
}

// Device buffers come from the device's stream-ordered memory pool (cudaMallocAsync on the
// grid's stream): a grid makes ~30 allocations, and plain cudaMalloc/cudaFree serialise
// across host threads, which bounded the request loop (every request creates a grid).  The
// pool keeps freed memory for reuse within this process (release threshold raised once);
// grid creation ends with a stream synchronisation, so its buffers are ready for any stream.
void pool_init_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------------------
// Host-side fault injection (error-path tests without a GPU fault): site k fails its n-th
// pass after arming, once, with the status the real call's failure gives.  Armed by
// tomo_inject_fault or, at the first check, by TOMO_FAULT="site:n[,site:n...]".
// ---------------------------------------------------------------------------------------
const char* const kFaultNames[FAULT_SITES] = {"alloc", "sync", "graph", "nan_input",
                                              "slow_request"};
std::atomic<long long> g_fault_left[FAULT_SITES];  // passes until the failure, 0 = disarmed

int fault_site(const char* name, size_t len) {
  for (int k = 0; k < FAULT_SITES; ++k)
    if (std::strlen(kFaultNames[k]) == len && std::strncmp(name, kFaultNames[k], len) == 0)
      return k;
  return -1;
}

void fault_env_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    const char* e = std::getenv("TOMO_FAULT");
    for (const char* c = e; c && *c;) {
      const char* colon = std::strchr(c, ':');
      if (!colon) break;
      const int k = fault_site(c, (size_t)(colon - c));
      char* end = nullptr;
      const long long n = std::strtoll(colon + 1, &end, 10);
      if (k >= 0 && n > 0) g_fault_left[k].store(n);
      c = (end && *end == ',') ? end + 1 : nullptr;
    }
  });
}

}  // namespace

bool tomo::fault_hit(FaultSite k) {
  fault_env_once();
  long long v = g_fault_left[k].load(std::memory_order_relaxed);
  while (v > 0) {
    if (g_fault_left[k].compare_exchange_weak(v, v - 1)) return v == 1;
  }
  return false;
}

namespace {

tomo_status dalloc(tomo_grid* G, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (fault_hit(FAULT_ALLOC))
    return fail(G, TOMO_ENOMEM, "injected device allocation failure (%zu bytes)", bytes);
  pool_init_once();
  CK(cudaMallocAsync(p, bytes, G->stream));
  G->dev_bytes += bytes;
  return TOMO_OK;
}

// Small pinned host blocks (the CG scalars and result scalars read back per solve) from
// 64 KiB page-locked slabs kept for the process: cudaMallocHost costs far more than a grid's
// other host work.
constexpr size_t kPinnedBlock = 256;
struct PinnedSlabs {
  std::mutex m;
  std::vector<void*> free_blocks;
};
PinnedSlabs& pinned_slabs() {
  static PinnedSlabs* s = new PinnedSlabs();  // never destroyed: blocks outlive static dtors
  return *s;
}

void* pinned_get(size_t bytes) {
  if (bytes > kPinnedBlock) return nullptr;
  PinnedSlabs& P = pinned_slabs();
  std::lock_guard<std::mutex> lk(P.m);
  if (P.free_blocks.empty()) {
    void* slab = nullptr;
    if (cudaMallocHost(&slab, 64 * 1024) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t o = 0; o < 64 * 1024; o += kPinnedBlock)
      P.free_blocks.push_back(static_cast<char*>(slab) + o);
  }
  void* b = P.free_blocks.back();
  P.free_blocks.pop_back();
  std::memset(b, 0, kPinnedBlock);
  return b;
}

void pinned_put(void* b) {
  if (!b) return;
  PinnedSlabs& P = pinned_slabs();
  std::lock_guard<std::mutex> lk(P.m);
  P.free_blocks.push_back(b);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller array; host arrays are copied into staging slot `slot`.
tomo_status stage_in(tomo_grid* G, const void* p, size_t bytes, int slot, const void** out,
                     bool* host) {
  *host = !is_device_ptr(p);
  if (!*host) {
    *out = p;
    return TOMO_OK;
  }
  if ((int)G->stage.size() <= slot) {
    G->stage.resize(slot + 1, nullptr);
    G->stage_size.resize(slot + 1, 0);
  }
  if (G->stage_size[slot] < bytes) {
    if (G->stage[slot]) cudaFreeAsync(G->stage[slot], G->stream);
    G->dev_bytes -= G->stage_size[slot];
    G->stage[slot] = nullptr;
    G->stage_size[slot] = 0;
    TRY(dalloc(G, &G->stage[slot], bytes));
    G->stage_size[slot] = bytes;
  }
  if (p) CK(cudaMemcpyAsync(G->stage[slot], p, bytes, cudaMemcpyHostToDevice, G->stream));
  *out = G->stage[slot];
  return TOMO_OK;
}

tomo_status stage_out(tomo_grid* G, void* p, size_t bytes, int slot, void** out, bool* host) {
  const void* o;
  *host = !is_device_ptr(p);
  if (!*host) {
    *out = p;
    return TOMO_OK;
  }
  if ((int)G->stage.size() <= slot) {
    G->stage.resize(slot + 1, nullptr);
    G->stage_size.resize(slot + 1, 0);
  }
  if (G->stage_size[slot] < bytes) {
    if (G->stage[slot]) cudaFreeAsync(G->stage[slot], G->stream);
    G->dev_bytes -= G->stage_size[slot];
    G->stage[slot] = nullptr;
    G->stage_size[slot] = 0;
    TRY(dalloc(G, &G->stage[slot], bytes));
    G->stage_size[slot] = bytes;
  }
  o = G->stage[slot];
  *out = const_cast<void*>(o);
  return TOMO_OK;
}

tomo_status copy_back(tomo_grid* G, void* host, const void* dev, size_t bytes, bool is_host) {
  if (!is_host) return TOMO_OK;
  CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, G->stream));
  return TOMO_OK;
}

// The grid's stream waits for a coarsest factorisation still running on the side stream.
tomo_status join_factor(tomo_grid* G) {
  if (!G->factor_pending) return TOMO_OK;
  G->factor_pending = false;
  CK(cudaStreamWaitEvent(G->stream, G->ev_factor, 0));
  return TOMO_OK;
}

tomo_status sync(tomo_grid* G) {
  TRY(join_factor(G));
  CK(cudaStreamSynchronize(G->stream));
  // (an injected failure is reported after the real synchronisation: no work is in flight)
  if (fault_hit(FAULT_SYNC)) return fail(G, TOMO_ECUDA, "injected stream synchronisation failure");
  return TOMO_OK;
}

// ---------------------------------------------------------------------------------------
// Profiling of fine-level matrix-free launches
// ---------------------------------------------------------------------------------------
tomo_status prof_begin(tomo_grid* G, cudaEvent_t* e0) {
  if (!G->prof) return TOMO_OK;
  if (G->ev_used + 2 > G->ev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      G->ev.push_back(e);
    }
  }
  *e0 = G->ev[G->ev_used];
  CK(cudaEventRecord(*e0, G->stream));
  return TOMO_OK;
}

tomo_status prof_end(tomo_grid* G, double bytes, int tag = -1) {
  if (!G->prof) return TOMO_OK;
  CK(cudaEventRecord(G->ev[G->ev_used + 1], G->stream));
  G->ev_used += 2;
  const size_t rec = G->ev_used / 2 - 1;
  if (G->ev_tag.size() <= rec) {
    G->ev_tag.resize(rec + 1);
    G->ev_bytes.resize(rec + 1);
    G->ev_iter.resize(rec + 1);
    G->ev_post.resize(rec + 1);
  }
  G->ev_tag[rec] = tag;
  G->ev_bytes[rec] = bytes;
  G->ev_iter[rec] = G->prof_iter;
  G->ev_post[rec] = G->prof_post ? 1 : 0;
  return TOMO_OK;
}

// After a host-issued solve that stopped at iteration itf: the launches it enqueued after
// the stop (the rest of iteration itf after its x/r update, and the iterations after it)
// returned at once on the device flag and did no work; they are left out of the timing.
void prof_drop_idle(tomo_grid* G, size_t rec0, int itf) {
  for (size_t q = rec0; q < G->ev_used / 2 && q < G->ev_tag.size(); ++q)
    if (G->ev_iter[q] > itf || (G->ev_iter[q] == itf && G->ev_post[q])) G->ev_tag[q] = -2;
}

// Level timing of one launch (kernel-timing mode): tag = level + 1.
struct LevelTimer {
  tomo_grid* G;
  int level;
  bool on;
  cudaEvent_t e0;
  LevelTimer(tomo_grid* g, int l) : G(g), level(l), on(g->prof) {
    if (on && prof_begin(G, &e0) != TOMO_OK) on = false;
  }
  ~LevelTimer() {
    if (on) prof_end(G, 0.0, level + 1);
  }
};

// Phase marks: 0 start, 1 filter+material, 2 level setup, 3 PCG, 4 sensitivity, 5 filter
// adjoints (gradient); 6 start, 7 end (OC step).
tomo_status pmark(tomo_grid* G, int i) {
  if (!G->phase_prof) return TOMO_OK;
  if (!G->phase_ev[i]) CK(cudaEventCreate(&G->phase_ev[i]));
  CK(cudaEventRecord(G->phase_ev[i], G->stream));
  return TOMO_OK;
}

tomo_status pcollect(tomo_grid* G, int first, int last) {
  if (!G->phase_prof) return TOMO_OK;
  CK(cudaEventSynchronize(G->phase_ev[last]));
  for (int i = first; i < last; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, G->phase_ev[i], G->phase_ev[i + 1]));
    G->phase_ms[i] += ms;
  }
  G->phase_calls += 1;
  return TOMO_OK;
}

template <typename T>
tomo_status march(tomo_grid* G, int level, int mode, MarchArgs<T> a, const T* s_override = nullptr) {
  const bool prof = G->prof && level == 0;
  cudaEvent_t e0;
  if (prof) TRY(prof_begin(G, &e0));
  std::unique_ptr<LevelTimer> lt;  // coarse levels: timed and binned by level
  if (G->prof && level > 0) lt.reset(new LevelTimer(G, level));
  a.g = G->L[level].g;
  a.s = s_override ? s_override : (const T*)G->L[level].s;
  a.mask = G->L[level].mask;
  a.partials = G->partials;
  a.counter = G->counter;
  int ctas = 0;
  bool fused_kernel = false;  // k_march2: the FP32 product/smoother the roofline reports
  if constexpr (sizeof(T) == 4) {
    if (a.xlo == nullptr) {
      fused_kernel = true;
      March2Args m{};
      m.g = a.g;
      m.s = a.s;
      m.mask = a.mask;
      m.x = a.x;
      m.b = a.b;
      m.xprev = a.xprev;
      m.y = a.y;
      m.c1 = a.c1;
      m.c2 = a.c2;
      m.partials = a.partials;
      m.counter = a.counter;
      m.sc = a.sc;
      m.dot_kind = a.dot_kind;
      m.skip = a.skip;
      m.xprev_zero = a.xprev_zero;
      m.tile_fixed = G->L[level].tile_fixed;
      m.invd = (const float*)G->L[level].invd;
      if (mode == M_CHEB && m.invd == nullptr)
        return fail(G, TOMO_EINVAL, "Chebyshev step on a level without its diagonal");
      if (a.gate != nullptr) return fail(G, TOMO_EINVAL, "gated product needs the FP64 path");
      March2Const k{(float)G->kinds.a0, (float)G->kinds.b0, (float)G->kinds.a7,
                    (float)G->kinds.b7, (float)G->kinds.ta, (float)G->kinds.tb,
                    (float)G->kinds.ua, (float)G->kinds.ud, (float)G->k0diag};
      CK(launch_march2(G->stream, mode, m, k, G->num_sms));
    } else {
      CK(launch_march<T>(G->stream, mode, a, elem_const<T>(G), G->num_sms, &ctas));
    }
  } else {
    CK(launch_march<T>(G->stream, mode, a, elem_const<T>(G), G->num_sms, &ctas));
  }
  G->launches += 1;
  if (prof && !fused_kernel && G->d.precision == TOMO_FP32) {
    // Level-0 launches of the generic kernel on the mixed path (FP64 residual replacement,
    // float-pair products) count toward level 0 but not toward the reported kernel.
    TRY(prof_end(G, 0.0, 1));
  } else if (prof) {
    const double nv = 3.0 * a.g.nn * sizeof(T);
    double bytes = nv + a.g.nel * (double)sizeof(T) + a.g.nn;  // x, s, mask
    if (a.xlo) bytes += nv;
    if (mode == M_APPLY) bytes += nv;                  // y
    else if (mode == M_RESID) bytes += 2 * nv;         // b, y
    else {
      bytes += ((a.c1 != T(0) && !a.xprev_zero) ? 3 : 2) * nv;  // b, (xprev), x_new
      if (fused_kernel) bytes += a.g.nn * (double)sizeof(T);       // D^-1 per node
    }
    TRY(prof_end(G, bytes));
  }
  return TOMO_OK;
}

// ---------------------------------------------------------------------------------------
// Multigrid hierarchy
// ---------------------------------------------------------------------------------------
template <typename T>
tomo_status setup_levels(tomo_grid* G) {
  if (G->s64) {
    CK(launch_convert<double, T>(G->stream, G->g.nel, (const T*)G->L[0].s, nullptr, G->s64));
    G->launches += 1;
  }
  for (size_t l = 1; l < G->L.size(); ++l) {
    CK(launch_coarsen_s<T>(G->stream, G->L[l - 1].g, G->L[l].g, (const T*)G->L[l - 1].s,
                           (T*)G->L[l].s));
    G->launches += 1;
  }
  for (auto& Lv : G->L) {
    if (!Lv.invd) continue;
    CK(launch_invdiag<T>(G->stream, Lv.g, (const T*)Lv.s, (T)G->k0diag, (T*)Lv.invd));
    G->launches += 1;
  }
  if (G->L.size() > 1) {
    // (a non-positive pivot is replaced by 1, which keeps the coarsest solve SPD; the
    // breakdown bit it sets is cleared when pcg_start resets the CG scalars: whether the
    // preconditioned CG converges is what the solve reports)
    auto& C = G->L.back();
    // one CTA for ~100+ us: overlapped with the first V-cycle's down-sweep, which needs it
    // only at the coarsest level (profiling keeps everything on one stream)
    TRY(join_factor(G));
    cudaStream_t fst = G->stream;
    if (!G->prof && G->side) {
      CK(cudaEventRecord(G->ev_fork, G->stream));
      CK(cudaStreamWaitEvent(G->side, G->ev_fork, 0));
      fst = G->side;
    }
    CK(launch_coarse_factor<T>(fst, C.g, (const T*)C.s, C.mask, dense_k0<T>(G),
                               (T*)G->coarseA, (T*)G->coarseD, &G->sc->status));
    G->launches += 1;
    if (fst != G->stream) {
      CK(cudaEventRecord(G->ev_factor, G->side));
      G->factor_pending = true;
    }
  }
  return TOMO_OK;
}

struct Cheb {
  double theta, delta, sigma;
};

Cheb cheb(const tomo_grid* G) {
  const double hi = G->lam_hi, lo = hi / G->cheb_ratio;
  Cheb c;
  c.theta = 0.5 * (hi + lo);
  c.delta = 0.5 * (hi - lo);
  c.sigma = c.theta / c.delta;
  return c;
}

// Chebyshev smoothing of K_l x = b on [lam_hi/ratio, lam_hi] of D^-1 K, degree K steps.
// zero_start: x_0 = 0 (first step needs no product).  On return *X holds the result.
int level_degree(const tomo_grid* G, int l) {
  return l == 0 ? G->d.smoother_degree : G->d.coarse_degree;
}



template <typename T>
tomo_status smooth(tomo_grid* G, int l, const T* b, T** X, T** Y, bool zero_start, bool dot,
                   const int* skip, bool first_done = false) {
  const Cheb cb = cheb(G);
  const int K = level_degree(G, l);
  const T k0d = (T)G->k0diag;
  auto& Lv = G->L[l];
  double rho_prev = 1.0 / cb.sigma;
  for (int s = 0; s < K; ++s) {
    const bool last = (s == K - 1);
    double c1, c2;
    if (s == 0) {
      c1 = 0.0;
      c2 = 1.0 / cb.theta;
    } else {
      const double rho = 1.0 / (2.0 * cb.sigma - rho_prev);
      c1 = rho * rho_prev;
      c2 = 2.0 * rho / cb.delta;
      rho_prev = rho;
    }
    const int dk = (dot && last) ? 2 : 0;
    if (s == 0 && zero_start) {
      if (!first_done) {  // (else the restriction or the CG update already wrote X)
        LevelTimer lt(G, l);
        CK(launch_jacobi<T>(G->stream, Lv.g, (const T*)Lv.s, Lv.mask, b, (T)c2, k0d, *X,
                            nullptr, G->partials, G->counter, G->sc, dk, skip));
        G->launches += 1;
      }
      // X = x1; x0 = 0 is implicit: the next step is told not to read Y
      continue;
    }
    MarchArgs<T> a{};
    a.x = *X;
    a.b = b;
    a.xprev = *Y;
    a.c1 = (T)c1;
    a.c2 = (T)c2;
    a.sc = G->sc;
    a.dot_kind = dk;
    a.skip = skip;
    a.xprev_zero = (s == 1 && zero_start) ? 1 : 0;
    TRY(march<T>(G, l, M_CHEB, a));
    std::swap(*X, *Y);
  }
  return TOMO_OK;
}

// Levels l .. coarsest of the V-cycle on b (level l's right-hand side) in one cluster
// launch (vtail.cu); first_done: level l's x already holds the zero-start step.
tomo_status vtail(tomo_grid* G, int l, const float* b, const int* skip, bool first_done) {
  TRY(join_factor(G));
  VTailArgs A{};
  const int nl = (int)G->L.size();
  A.nlev = nl - l;
  A.first_done = first_done ? 1 : 0;
  A.nc = G->coarse_n;
  A.ld = G->vt_ld;
  A.Ainv = (const float*)G->coarseA;
  A.dsc = (const float*)G->coarseD;
  A.eb = (float*)G->vt_eb;
  A.skip = skip;
  const Cheb cb = cheb(G);
  for (int q = 0; q < A.nlev; ++q) {
    const tomo_level& Lv = G->L[l + q];
    VTailLevel& V = A.L[q];
    V.g = Lv.g;
    V.s = (const float*)Lv.s;
    V.mask = Lv.mask;
    V.invd = (const float*)Lv.invd;
    V.x = (float*)Lv.x;
    V.xp = (float*)Lv.xp;
    V.b = q == 0 ? const_cast<float*>(b) : (float*)Lv.b;
    V.t = (float*)Lv.t;
    V.K = level_degree(G, l + q);
    if (V.K > kVtMaxDeg) return fail(G, TOMO_EINVAL, "coarse tail: degree above %d", kVtMaxDeg);
    double rho_prev = 1.0 / cb.sigma;
    for (int s = 0; s < V.K; ++s) {  // the coefficients smooth() uses
      if (s == 0) {
        V.c1[s] = 0.0f;
        V.c2[s] = (float)(1.0 / cb.theta);
      } else {
        const double rho = 1.0 / (2.0 * cb.sigma - rho_prev);
        V.c1[s] = (float)(rho * rho_prev);
        V.c2[s] = (float)(2.0 * rho / cb.delta);
        rho_prev = rho;
      }
    }
  }
  LevelTimer lt(G, l);
  CK(launch_vtail(G->stream, A, elem_const<float>(G)));
  G->launches += 1;
  return TOMO_OK;
}

// z = V-cycle(b) on level l; *out receives the buffer holding z.
template <typename T>
tomo_status vcycle(tomo_grid* G, int l, const T* b, T** out, bool dot, const int* skip,
                   bool first_done = false) {
  auto& Lv = G->L[l];
  const int nl = (int)G->L.size();
  if (l == nl - 1) {
    TRY(join_factor(G));
    LevelTimer lt(G, l);
    CK(launch_coarse_apply<T>(G->stream, G->coarse_n, (const T*)G->coarseA,
                              (const T*)G->coarseD, b, (T*)Lv.x, skip));
    G->launches += 1;
    *out = (T*)Lv.x;
    return TOMO_OK;
  }
  if constexpr (sizeof(T) == 4) {
    if (G->vt_on && l == G->vt_level && l > 0 && (G->wlevels >> l) == 0u) {
      // levels l .. coarsest in one cluster launch (the same operator as the launched
      // levels below; ping-pong as smooth(): 2K - 1 swaps leave the result in xp)
      TRY(vtail(G, l, b, skip, first_done));
      *out = (T*)((2 * level_degree(G, l) - 1) % 2 ? Lv.xp : Lv.x);
      return TOMO_OK;
    }
  }
  T* X = (T*)Lv.x;
  T* Y = (T*)Lv.xp;
  TRY(smooth<T>(G, l, b, &X, &Y, true, false, skip, first_done));
  {
    MarchArgs<T> a{};
    a.x = X;
    a.b = b;
    a.y = (T*)Lv.t;
    a.skip = skip;
    TRY(march<T>(G, l, M_RESID, a));
  }
  auto& Lc = G->L[l + 1];
  // the first Chebyshev step of the next level (from zero) is pointwise: fuse it here
  const bool fuse = (l + 1 < nl - 1);
  const Cheb cb = cheb(G);
  {
  LevelTimer lt(G, l);
  CK(launch_restrict<T>(G->stream, Lv.g, Lc.g, (const T*)Lv.t, (T*)Lc.b, Lc.mask, skip,
                        fuse ? (T*)Lc.x : nullptr, (const T*)Lc.s, (T)(1.0 / cb.theta),
                        (T)G->k0diag));
  G->launches += 1;
  }
  T* zc = nullptr;
  TRY(vcycle<T>(G, l + 1, (const T*)Lc.b, &zc, false, skip, fuse));
  {
    LevelTimer lt(G, l);
    CK(launch_prolong_add<T>(G->stream, Lv.g, Lc.g, zc, X, Lv.mask, skip));
  }
  G->launches += 1;
  if (((G->wlevels >> l) & 1u) && l + 2 < nl) {
    // W-cycle at this level: a second coarse-grid correction from the corrected iterate
    // (x += P M_c P^T (b - A x); symmetric, so the cycle stays an SPD preconditioner); the
    // level above the coarsest is left out (its exact coarse solve leaves nothing to correct)
    MarchArgs<T> a{};
    a.x = X;
    a.b = b;
    a.y = (T*)Lv.t;
    a.skip = skip;
    TRY(march<T>(G, l, M_RESID, a));
    {
      LevelTimer lt(G, l);
      CK(launch_restrict<T>(G->stream, Lv.g, Lc.g, (const T*)Lv.t, (T*)Lc.b, Lc.mask, skip,
                            fuse ? (T*)Lc.x : nullptr, (const T*)Lc.s, (T)(1.0 / cb.theta),
                            (T)G->k0diag));
      G->launches += 1;
    }
    TRY(vcycle<T>(G, l + 1, (const T*)Lc.b, &zc, false, skip, fuse));
    {
      LevelTimer lt(G, l);
      CK(launch_prolong_add<T>(G->stream, Lv.g, Lc.g, zc, X, Lv.mask, skip));
    }
    G->launches += 1;
  }
  TRY(smooth<T>(G, l, b, &X, &Y, false, dot, skip));
  *out = X;
  return TOMO_OK;
}

// z = M r with rz/beta from the fused dot
template <typename T>
tomo_status precond(tomo_grid* G, const T* r, T** z, bool first_done0 = false) {
  const int* skip = &G->sc->done;
  if (G->d.precond == TOMO_PRECOND_JACOBI) {
    auto& L0 = G->L[0];
    CK(launch_jacobi<T>(G->stream, L0.g, (const T*)L0.s, L0.mask, r, T(1), (T)G->k0diag,
                        (T*)L0.x, nullptr, G->partials, G->counter, G->sc, 2, skip));
    G->launches += 1;
    *z = (T*)L0.x;
    return TOMO_OK;
  }
  return vcycle<T>(G, 0, r, z, true, skip, first_done0);
}

// One PCG iteration: q = A p (alpha), x/r update (convergence test), residual replacement
// when it % rr_every == 0 (decided on the device), z = M r (beta), p = z + beta p.  Every
// kernel returns at once when the device flag sc->done is set.
template <typename T>
tomo_status enqueue_iteration(tomo_grid* G) {
  const int n = 3 * G->g.nn;
  T* r = (T*)G->r;
  T* p = (T*)G->p;
  T* q = (T*)G->q;
  T* xhi = (T*)G->xhi;
  T* xlo = G->prec == TOMO_FP32 ? (T*)G->xlo : nullptr;
  MarchArgs<T> a{};
  a.x = p;
  a.y = q;
  a.sc = G->sc;
  a.dot_kind = 1;
  a.skip = &G->sc->done;
  TRY(march<T>(G, 0, M_APPLY, a));
  // fused grids: the update also writes the next V-cycle's first finest-level step
  T* x1 = G->fuse_j0 ? (T*)G->L[0].x : nullptr;
  const T c2 = (T)(1.0 / cheb(G).theta);
  CK(launch_cg_xr<T>(G->stream, n, xhi, xlo, r, p, q, G->partials, G->counter, G->sc, x1,
                     (const T*)G->invd, c2));
  G->launches += 1;
  G->prof_post = true;  // the convergence test of this iteration is enqueued
  if (G->d.rr_every > 0) {
    // residual replacement r = f - K x on iterations it % rr_every == 0 (device gate), in
    // FP64 for both precisions
    if constexpr (sizeof(T) == 8) {
      MarchArgs<T> rr{};
      rr.x = xhi;
      rr.b = (const T*)G->rhs64;
      rr.y = r;
      rr.skip = &G->sc->done;
      rr.gate = G->sc;
      TRY(march<T>(G, 0, M_RESID, rr));
    } else {
      // one launch: the float-pair iterate is joined into double on load, the FP64
      // residual is rounded to float on store
      MarchArgs<double> rr{};
      rr.xf_hi = xhi;
      rr.xf_lo = xlo;
      rr.b = G->rhs64;
      rr.yf = r;
      rr.skip = &G->sc->done;
      rr.gate = G->sc;
      if (G->fuse_j0) {  // the first step follows the replaced residual
        rr.x1f = (float*)x1;
        rr.invdf = (const float*)G->invd;
        rr.c2f = (float)c2;
      }
      TRY(march<double>(G, 0, M_RESID, rr, G->s64));
    }
  }
  T* z = nullptr;
  TRY(precond<T>(G, r, &z, G->fuse_j0));
  if (G->cond_capture)  // the device-side loop: this launch also decides the next iteration
    CK(launch_cg_p_cond<T>(G->stream, n, p, z, G->sc, G->cond_handle, G->counter + 3));
  else
    CK(launch_cg_p<T>(G->stream, n, p, z, G->sc));
  G->launches += 1;
  return TOMO_OK;
}

// Capture one iteration into the body of a conditional-while graph node; the body ends
// with a kernel that clears the condition once CG has stopped.
template <typename T>
tomo_status build_loop_graph(tomo_grid* G, cudaGraphExec_t* out) {
  TRY(join_factor(G));  // (nothing outside the capture may be waited on inside it)
  if (!G->cap_stream) CK(cudaStreamCreateWithFlags(&G->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    CK(e);
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t saved = G->stream;
  G->stream = G->cap_stream;
  e = cudaStreamBeginCaptureToGraph(G->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  tomo_status st = TOMO_OK;
  const int64_t before = G->launches;
  if (e == cudaSuccess) {
    // the iteration's last kernel (the p update) also runs the loop test
    G->cond_capture = true;
    G->cond_handle = h;
    st = enqueue_iteration<T>(G);
    G->cond_capture = false;
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(G->stream, &captured);
    if (st == TOMO_OK && e3 != cudaSuccess) e = e3;
  }
  G->stream = saved;
  G->iter_launches = G->launches - before;  // captured, not executed
  G->launches = before;
  if (e != cudaSuccess || st != TOMO_OK) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != TOMO_OK) return st;
    CK(e);
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  return TOMO_OK;
}

// Preconditioned CG on K(s_0) x = f.  x (xhi [+ xlo]) holds the start on entry (warm) or is
// zeroed (cold).  The iteration loop runs on the device (conditional-while graph); with
// profiling enabled it is issued from the host in batches instead, so that every launch
// can be bracketed by events.
// pcg up to the loop: scalars, start iterate, r = f - K x (or f), p = 0.  *trivial: the
// load is zero, the solution (0) and info are already final.
template <typename T>
tomo_status pcg_start(tomo_grid* G, bool warm, tomo_solve_info* info, bool* trivial) {
  *trivial = false;
  const Geom g = G->g;
  const int n = 3 * g.nn;
  T* r = (T*)G->r;
  T* p = (T*)G->p;
  T* xhi = (T*)G->xhi;
  T* xlo = G->prec == TOMO_FP32 ? (T*)G->xlo : nullptr;
  const double ff = G->rhs_ff;
  const double rtol = G->d.rtol;
  CgScalars h{};
  h.ff = ff;
  h.tol2 = rtol * rtol * ff;
  h.maxit = G->d.maxit;
  h.rr_every = G->d.rr_every > 0 ? G->d.rr_every : 0;
  *G->h_sc = h;
  if (ff == 0.0) {
    CK(launch_cg_start<T>(G->stream, n, xhi, xlo, nullptr, nullptr, G->sc, h));
    G->launches += 1;
    TRY(sync(G));
    if (info) {
      info->iters = 0;
      info->rel_res = 0.0;
      info->status = TOMO_OK;
      info->mg_levels = (int)G->L.size();
    }
    G->have_solution = true;
    *trivial = true;
    return TOMO_OK;
  }
  if (warm) {
    CK(launch_cg_start<T>(G->stream, n, nullptr, nullptr, nullptr, p, G->sc, h));
    G->launches += 1;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (G->s64) {  // r = f - K x evaluated in FP64 from the float pair, rounded once
        MarchArgs<double> rr{};
        rr.xf_hi = xhi;
        rr.xf_lo = xlo;
        rr.b = G->rhs64;
        rr.yf = r;
        TRY(march<double>(G, 0, M_RESID, rr, G->s64));
        done = true;
      }
    }
    if (!done) {
      MarchArgs<T> a{};
      a.x = xhi;
      a.xlo = xlo;
      a.b = (const T*)G->rhs_T;
      a.y = r;
      TRY(march<T>(G, 0, M_RESID, a));
    }
  } else if (G->rhs_id == 0) {  // x = 0, p = 0, r = f: zeros, then the load's nonzero entries
    CK(launch_cg_start<T>(G->stream, n, xhi, xlo, r, p, G->sc, h));
    CK(launch_scatter_vec<T>(G->stream, G->load_nnz, G->load_idx, G->load_val, r));
    G->launches += 2;
  } else {
    CK(launch_cg_start<T>(G->stream, n, xhi, xlo, nullptr, p, G->sc, h));
    CK(launch_mask_copy<T>(G->stream, g, (const T*)G->rhs_T, G->L[0].mask, r));
    G->launches += 2;
  }
  return TOMO_OK;
}

// Status and info of a finished loop from the host copy of the scalars (G->h_sc).
tomo_status pcg_result(tomo_grid* G, tomo_solve_info* info) {
  const double ff = G->rhs_ff;
  const CgScalars& hs = *G->h_sc;
  tomo_status st = TOMO_OK;
  if (hs.status & DEV_TIMEOUT) {
    // a bounded device wait ran out mid-iteration: the iterate is not a solution
    if (info) {
      info->iters = hs.it;
      info->rel_res = std::sqrt(std::max(hs.rr, 0.0) / ff);
      info->status = TOMO_ETIMEOUT;
      info->mg_levels = (int)G->L.size();
    }
    G->have_solution = false;
    // the stopped launch can leave a block-reduction counter mid-count: zero it for the
    // next solve (stream order: after the loop)
    if (cudaMemsetAsync(G->counter, 0, sizeof(unsigned) * 4, G->stream) != cudaSuccess)
      cudaGetLastError();
    return fail(G, TOMO_ETIMEOUT, "a device wait ran out at CG iteration %d", hs.it);
  }
  if (hs.status & DEV_NAN) st = TOMO_ENAN;
  else if (hs.status & DEV_BREAKDOWN) st = TOMO_ENOCONV;
  else if (hs.rr > hs.tol2) st = TOMO_ENOCONV;
  if (info) {
    info->iters = hs.it;
    info->rel_res = std::sqrt(std::max(hs.rr, 0.0) / ff);
    info->status = st;
    info->mg_levels = (int)G->L.size();
  }
  G->have_solution = true;
  if (st == TOMO_ENAN) return fail(G, st, "NaN/Inf in the CG iteration at iteration %d", hs.it);
  if (st == TOMO_ENOCONV)
    return fail(G, st, "CG stopped after %d iterations at relative residual %.3e%s", hs.it,
                std::sqrt(std::max(hs.rr, 0.0) / ff),
                (hs.status & DEV_BREAKDOWN) ? " (breakdown)" : "");
  return TOMO_OK;
}

tomo_status set_smoother(tomo_grid* G, int fine, int coarse, double ratio, double lam,
                         int64_t wlevels = -1);

template <typename T>
tomo_status pcg_once(tomo_grid* G, bool warm, tomo_solve_info* info) {
  bool trivial = false;
  TRY(pcg_start<T>(G, warm, info, &trivial));
  if (trivial) return TOMO_OK;
  const int n = 3 * G->g.nn;
  T* r = (T*)G->r;
  T* p = (T*)G->p;
  T* z = nullptr;
  TRY(precond<T>(G, r, &z));
  CK(launch_cg_p<T>(G->stream, n, p, z, G->sc));
  G->launches += 1;
  cudaGraphExec_t& exec = G->rhs_id == 0 ? G->loop_exec : G->loop_exec_adj;
  if (G->use_graph && !G->prof && !exec) {
    if (build_loop_graph<T>(G, &exec) != TOMO_OK) {
      // the device-side loop could not be captured: issue the iterations from the host
      cudaGetLastError();
      G->use_graph = false;
      G->err.clear();
    }
  }
  if (G->use_graph && !G->prof) {
    if (fault_hit(FAULT_GRAPH)) return fail(G, TOMO_ECUDA, "injected CG loop launch failure");
    CK(cudaGraphLaunch(exec, G->stream));
    CK(cudaMemcpyAsync(G->h_sc, G->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, G->stream));
    TRY(sync(G));
    G->launches += (int64_t)G->h_sc->loops * G->iter_launches;
  } else {
    const int batch = 4;
    int it = 0;
    bool done = false;
    const size_t rec0 = G->ev_used / 2;
    while (!done) {
      for (int b2 = 0; b2 < batch; ++b2, ++it) {
        G->prof_iter = it + 1;
        G->prof_post = false;
        const tomo_status se = enqueue_iteration<T>(G);
        if (se != TOMO_OK) {
          G->prof_iter = 0;
          return se;
        }
      }
      G->prof_iter = 0;
      CK(cudaMemcpyAsync(G->h_sc, G->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, G->stream));
      TRY(sync(G));
      done = G->h_sc->done != 0;
      if (it > G->d.maxit + batch) done = true;
    }
    if (G->prof) prof_drop_idle(G, rec0, G->h_sc->it);
  }
  return pcg_result(G, info);
}

// The solve, and with `fallback` a second chance: a smoothing interval whose upper end lies
// below the spectrum of D^-1 K (a tuned bound on a design it does not fit) can make the
// V-cycle indefinite (r^T z <= 0 stops CG) or slow; the solve is then redone from zero at
// the element bound, which always holds, and the grid keeps that bound.
template <typename T>
tomo_status pcg(tomo_grid* G, bool warm, tomo_solve_info* info, bool fallback = true) {
  NvtxRange range("tomo: PCG (S3-S5)");
  tomo_status st = pcg_once<T>(G, warm, info);
  if (st == TOMO_OK || !fallback || st == TOMO_ECUDA || st == TOMO_EINVAL ||
      G->d.precond != TOMO_PRECOND_MG || !(G->lam_hi < G->lam_bound))
    return st;
  G->bound_fallbacks += 1;
  TRY(set_smoother(G, G->d.smoother_degree, G->d.coarse_degree, G->cheb_ratio, G->lam_bound));
  G->err.clear();
  return pcg_once<T>(G, false, info);
}

// dV/dz = P^T v with v_e = h^3 (Section III-D), written to out.
template <typename T>
tomo_status volume_gradient(tomo_grid* G, T* out) {
  const int ne = G->g.nel;
  if (G->dvdz_ready) {  // design independent: computed on the first call, copied after
    CK(cudaMemcpyAsync(out, G->dvdz, sizeof(T) * ne, cudaMemcpyDeviceToDevice, G->stream));
    return TOMO_OK;
  }
  CK(launch_fill<T>(G->stream, ne, (T*)G->dvdz, (T)(G->d.h * G->d.h * G->d.h)));
  CK(launch_filter<T>(G->stream, G->g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                      G->filter_radius,
                      (const T*)G->dvdz, (const T*)G->Hs, out, 1, 0, T(0), T(0), T(0), T(0),
                      nullptr));
  CK(cudaMemcpyAsync(G->dvdz, out, sizeof(T) * ne, cudaMemcpyDeviceToDevice, G->stream));
  G->launches += 2;
  G->dvdz_ready = true;
  return TOMO_OK;
}

template <typename T>
T* x_lo(tomo_grid* G) {
  return G->prec == TOMO_FP32 ? (T*)G->xlo : nullptr;
}

tomo_status check_prec(tomo_grid* G, bool want64) {
  if (!G) return TOMO_EINVAL;
  if ((G->prec == TOMO_FP64) != want64)
    return fail(G, TOMO_EINVAL, "entry point precision does not match the grid (%s grid)",
                G->prec == TOMO_FP64 ? "FP64" : "FP32");
  return TOMO_OK;
}

// ---------------------------------------------------------------------------------------
// Entry point bodies
// ---------------------------------------------------------------------------------------
template <typename T>
tomo_status do_filter(tomo_grid* G, const T* in, T* out, int transpose) {
  if (!in || !out) return fail(G, TOMO_EINVAL, "null array");
  const size_t bytes = sizeof(T) * (size_t)G->g.nel;
  const void* din;
  void* dout;
  bool hin, hout;
  TRY(stage_in(G, in, bytes, 0, &din, &hin));
  TRY(stage_out(G, out, bytes, 1, &dout, &hout));
  if (din == dout) return fail(G, TOMO_EINVAL, "in and out overlap");
  CK(launch_filter<T>(G->stream, G->g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                      G->filter_radius, (const T*)din,
                      (const T*)G->Hs, (T*)dout, transpose ? 1 : 0, 0, T(0), T(0), T(0), T(0),
                      nullptr));
  G->launches += 1;
  TRY(copy_back(G, out, dout, bytes, hout));
  if (hin || hout) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_coarse_grain(tomo_grid* G, const T* z, int nb, T* zc) {
  if (!z || !zc) return fail(G, TOMO_EINVAL, "null array");
  if (nb < 1) return fail(G, TOMO_EINVAL, "block size must be >= 1 (got %d)", nb);
  const Geom& g = G->g;
  const size_t nc = (size_t)((g.nx + nb - 1) / nb) * ((g.ny + nb - 1) / nb) *
                    ((g.nz + nb - 1) / nb);
  const void* dz;
  void* dzc;
  bool hin, hout;
  TRY(stage_in(G, z, sizeof(T) * (size_t)g.nel, 0, &dz, &hin));
  TRY(stage_out(G, zc, sizeof(T) * nc, 1, &dzc, &hout));
  if (dz == dzc) return fail(G, TOMO_EINVAL, "z and z_coarse overlap");
  CK(launch_coarse_grain<T>(G->stream, g, nb, (const T*)dz, (T*)dzc));
  G->launches += 1;
  TRY(copy_back(G, zc, dzc, sizeof(T) * nc, hout));
  if (hin || hout) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_apply(tomo_grid* G, const T* rho, const T* x, T* y) {
  if (!rho || !x || !y) return fail(G, TOMO_EINVAL, "null array");
  const size_t be = sizeof(T) * (size_t)G->g.nel, bn = sizeof(T) * 3 * (size_t)G->g.nn;
  const void *drho, *dx;
  void* dy;
  bool h1, h2, h3;
  TRY(stage_in(G, rho, be, 0, &drho, &h1));
  TRY(stage_in(G, x, bn, 2, &dx, &h2));
  TRY(stage_out(G, y, bn, 3, &dy, &h3));
  if (dx == dy) return fail(G, TOMO_EINVAL, "x and y overlap");
  const tomo_grid_desc& d = G->d;
  CK(launch_material<T>(G->stream, G->g.nel, (const T*)drho, (T)d.E0, (T)d.Emin, (T)d.penal,
                        (T)d.h, (T*)G->L[0].s));
  G->launches += 1;
  // the product sees masked input: fixed entries of x are ignored
  T* xm = (T*)G->q;
  CK(launch_mask_copy<T>(G->stream, G->g, (const T*)dx, G->L[0].mask, xm));
  G->launches += 1;
  MarchArgs<T> a{};
  a.x = xm;
  a.y = (T*)dy;
  TRY(march<T>(G, 0, M_APPLY, a));
  TRY(copy_back(G, y, dy, bn, h3));
  if (h1 || h2 || h3) TRY(sync(G));
  return TOMO_OK;
}

// r = f - K(rho) (u + ulo) on the free DOFs, by the product kernel's residual mode with the
// pair input (FP32 grids) or plain input (FP64 grids).
template <typename T>
tomo_status do_residual(tomo_grid* G, const T* rho, const T* u, const T* ulo, T* r) {
  if (!rho || !u || !r) return fail(G, TOMO_EINVAL, "null array");
  if (ulo && G->prec == TOMO_FP64) return fail(G, TOMO_EINVAL, "u_lo is for FP32 grids");
  const size_t be = sizeof(T) * (size_t)G->g.nel, bn = sizeof(T) * 3 * (size_t)G->g.nn;
  const void *drho, *du, *dul = nullptr;
  void* dr;
  bool h1, h2, h3 = false, h4;
  TRY(stage_in(G, rho, be, 0, &drho, &h1));
  TRY(stage_in(G, u, bn, 2, &du, &h2));
  if (ulo) TRY(stage_in(G, ulo, bn, 6, &dul, &h3));
  TRY(stage_out(G, r, bn, 3, &dr, &h4));
  const tomo_grid_desc& d = G->d;
  CK(launch_material<T>(G->stream, G->g.nel, (const T*)drho, (T)d.E0, (T)d.Emin, (T)d.penal,
                        (T)d.h, (T*)G->L[0].s));
  G->launches += 1;
  // masked copies: fixed entries of u are ignored
  T* xm = (T*)G->q;
  T* xl = (T*)G->p;
  CK(launch_mask_copy<T>(G->stream, G->g, (const T*)du, G->L[0].mask, xm));
  G->launches += 1;
  if (dul) {
    CK(launch_mask_copy<T>(G->stream, G->g, (const T*)dul, G->L[0].mask, xl));
    G->launches += 1;
  }
  MarchArgs<T> a{};
  a.x = xm;
  a.xlo = dul ? xl : nullptr;
  a.b = (const T*)G->f_T;
  a.y = (T*)dr;
  TRY(march<T>(G, 0, M_RESID, a));
  TRY(copy_back(G, r, dr, bn, h4));
  if (h1 || h2 || h3 || h4) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_solve(tomo_grid* G, const T* rho, T* u, tomo_solve_info* info) {
  if (!rho || !u) return fail(G, TOMO_EINVAL, "null array");
  const size_t be = sizeof(T) * (size_t)G->g.nel, bn = sizeof(T) * 3 * (size_t)G->g.nn;
  const void *drho = nullptr, *du = nullptr;
  bool h1, h2;
  TRY(stage_in(G, rho, be, 0, &drho, &h1));
  TRY(stage_in(G, u, bn, 2, &du, &h2));
  const tomo_grid_desc& d = G->d;
  CK(launch_material<T>(G->stream, G->g.nel, (const T*)drho, (T)d.E0, (T)d.Emin, (T)d.penal,
                        (T)d.h, (T*)G->L[0].s));
  G->launches += 1;
  TRY(setup_levels<T>(G));
  CK(launch_mask_copy<T>(G->stream, G->g, (const T*)du, G->L[0].mask, (T*)G->xhi));
  G->launches += 1;
  if (x_lo<T>(G)) CK(cudaMemsetAsync(G->xlo, 0, bn, G->stream));
  tomo_status st = pcg<T>(G, true, info);
  if (st != TOMO_OK && st != TOMO_ENOCONV && st != TOMO_ENAN) return st;
  // u = x (pair summed)
  void* dout;
  bool hout;
  TRY(stage_out(G, u, bn, 3, &dout, &hout));
  CK(launch_convert<T, T>(G->stream, 3 * G->g.nn, (const T*)G->xhi, (const T*)x_lo<T>(G),
                          (T*)dout));
  G->launches += 1;
  TRY(copy_back(G, u, dout, bn, hout));
  TRY(sync(G));
  return st;
}

template <typename T>
tomo_status compliance_and_sens(tomo_grid* G, const T* drho, const T* du, const T* dulo,
                                double* compliance, T* ddc) {
  const tomo_grid_desc& d = G->d;
  if (compliance) {
    // f^T u: the load is sparse (point, line, face loads), so only its nonzero entries
    if (G->load_nnz <= (1 << 18)) {
      CK(launch_sparse_dot<T>(G->stream, G->load_nnz, G->load_idx, G->load_val, du, dulo,
                              G->partials, G->counter, G->dscal));
    } else {
      CK(launch_dot<double, T>(G->stream, 3 * G->g.nn, G->f64, du, dulo, G->partials,
                               G->counter, G->dscal));
    }
    G->launches += 1;
  }
  if (ddc) {
    CK(launch_sensitivity<T>(G->stream, G->g, drho, du, dulo, nullptr, nullptr,
                             elem_const<T>(G), (T)d.penal,
                             (T)d.E0, (T)d.Emin, (T)d.h, ddc));
    G->launches += 1;
  }
  return TOMO_OK;
}

tomo_status write_scalar(tomo_grid* G, double* dst, const double* dev_src) {
  if (!dst) return TOMO_OK;
  if (is_device_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, dev_src, sizeof(double), cudaMemcpyDeviceToDevice, G->stream));
    return TOMO_OK;
  }
  CK(cudaMemcpyAsync(G->h_scal, dev_src, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
  TRY(sync(G));
  *dst = *G->h_scal;
  return TOMO_OK;
}

template <typename T>
tomo_status do_sensitivity(tomo_grid* G, const T* rho, const T* u, double* compliance, T* dc) {
  if (!rho || !u) return fail(G, TOMO_EINVAL, "null array");
  const size_t be = sizeof(T) * (size_t)G->g.nel, bn = sizeof(T) * 3 * (size_t)G->g.nn;
  const void *drho = nullptr, *du = nullptr;
  void* ddc = nullptr;
  bool h1, h2, h3 = false;
  TRY(stage_in(G, rho, be, 0, &drho, &h1));
  TRY(stage_in(G, u, bn, 2, &du, &h2));
  if (dc) TRY(stage_out(G, dc, be, 1, &ddc, &h3));
  TRY(compliance_and_sens<T>(G, (const T*)drho, (const T*)du, nullptr, compliance, (T*)ddc));
  if (dc) TRY(copy_back(G, dc, ddc, be, h3));
  TRY(write_scalar(G, compliance, G->dscal));
  if (h1 || h2 || h3) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_oc(tomo_grid* G, const T* z, const T* dcdz, const T* dvdz, double volfrac,
                  double move, T* znew, double* change) {
  NvtxRange range("tomo: OC update (Section III-D)");
  if (!z || !dcdz || !dvdz || !znew) return fail(G, TOMO_EINVAL, "null array");
  if (!(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0))
    return fail(G, TOMO_EINVAL, "volfrac must be in (0,1] and move > 0");
  const size_t be = sizeof(T) * (size_t)G->g.nel;
  const void *dz, *ddc, *dw;
  void* dzn;
  bool h1, h2, h3, h4;
  TRY(stage_in(G, z, be, 0, &dz, &h1));
  TRY(stage_in(G, dcdz, be, 1, &ddc, &h2));
  TRY(stage_in(G, dvdz, be, 4, &dw, &h3));
  TRY(stage_out(G, znew, be, 5, &dzn, &h4));
  if (dzn == dz || dzn == ddc || dzn == dw) return fail(G, TOMO_EINVAL, "z_new overlaps an input");
  const double vmax = volfrac * (double)G->g.nel * G->d.h * G->d.h * G->d.h;
  TRY(pmark(G, 6));
  CK(launch_oc<T>(G->stream, G->g.nel, (const T*)dz, (const T*)ddc, (const T*)dw, vmax, move,
                  (T*)dzn, G->partials, G->counter, G->dscal + 2, G->dscal + 1,
                  oc_max_blocks(G->g.nel)));
  G->launches += (sizeof(T) == 8) ? 11 : 10;
  TRY(pmark(G, 7));
  if (G->phase_prof) {
    CK(cudaEventSynchronize(G->phase_ev[7]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, G->phase_ev[6], G->phase_ev[7]));
    G->phase_ms[6] += ms;
  }
  TRY(copy_back(G, znew, dzn, be, h4));
  TRY(write_scalar(G, change, G->dscal + 1));
  if (h1 || h2 || h3 || h4) TRY(sync(G));
  return TOMO_OK;
}

// Arrays of one gradient evaluation (device pointers of staged host arrays).
struct GradIO {
  const void* dz = nullptr;
  void* ddc = nullptr;
  void* ddv = nullptr;
  bool h1 = false, h2 = false, h3 = false;
};

// S1-S2 of a gradient: stage the arrays, rho = P z, s = h E(rho), coarse moduli and the
// coarsest factorisation.
template <typename T>
tomo_status gradient_begin(tomo_grid* G, const T* z, T* dcdz, T* dvdz, GradIO* io) {
  NvtxRange range("tomo: filter, material, levels (S1-S2)");
  if (!z || !dcdz) return fail(G, TOMO_EINVAL, "null array");
  const size_t be = sizeof(T) * (size_t)G->g.nel;
  const tomo_grid_desc& d = G->d;
  TRY(stage_in(G, z, be, 0, &io->dz, &io->h1));
  TRY(stage_out(G, dcdz, be, 1, &io->ddc, &io->h2));
  if (dvdz) TRY(stage_out(G, dvdz, be, 4, &io->ddv, &io->h3));
  const void* dz = io->dz;
  T* rho = (T*)G->rho;
  TRY(pmark(G, 0));
  // S1: rho = P z, s = h (Emin + rho^p (E0 - Emin))
  CK(launch_filter<T>(G->stream, G->g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                      G->filter_radius, (const T*)dz,
                      (const T*)G->Hs, rho, 0, 1, (T)d.E0, (T)d.Emin, (T)d.penal, (T)d.h,
                      (T*)G->L[0].s));
  G->launches += 1;
  if (fault_hit(FAULT_NAN))  // injected: element 0's modulus becomes NaN (all bits set)
    CK(cudaMemsetAsync(G->L[0].s, 0xFF, sizeof(T), G->stream));
  TRY(pmark(G, 1));
  // S2: coarse moduli, coarsest factorisation
  TRY(setup_levels<T>(G));
  TRY(pmark(G, 2));
  return TOMO_OK;
}

// S6-S7 of a gradient after the solve: compliance, dc/drho, dc/dz = P^T dc/drho, dV/dz.
// defer_scalar: a host `compliance` is left in G->h_scal (copied asynchronously; the caller
// synchronises the stream and reads it) instead of synchronising here.
template <typename T>
tomo_status gradient_end(tomo_grid* G, const GradIO& io, double* compliance, T* dcdz, T* dvdz,
                         bool defer_scalar = false) {
  NvtxRange range("tomo: compliance, sensitivities, filter adjoint (S6-S7)");
  const size_t be = sizeof(T) * (size_t)G->g.nel;
  T* rho = (T*)G->rho;
  void* ddc = io.ddc;
  void* ddv = io.ddv;
  // S6: compliance and dc/drho
  TRY(compliance_and_sens<T>(G, rho, (const T*)G->xhi, (const T*)x_lo<T>(G), compliance,
                             (T*)G->dcp));
  TRY(pmark(G, 4));
  // S7: dc/dz = P^T dc/drho, dV/dz = P^T v
  CK(launch_filter<T>(G->stream, G->g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                      G->filter_radius,
                      (const T*)G->dcp, (const T*)G->Hs, (T*)ddc, 1, 0, T(0), T(0), T(0), T(0),
                      nullptr));
  G->launches += 1;
  if (ddv) TRY(volume_gradient<T>(G, (T*)ddv));
  TRY(pmark(G, 5));
  TRY(pcollect(G, 0, 5));
  TRY(copy_back(G, dcdz, ddc, be, io.h2));
  if (dvdz) TRY(copy_back(G, dvdz, ddv, be, io.h3));
  if (defer_scalar && compliance && !is_device_ptr(compliance))
    CK(cudaMemcpyAsync(G->h_scal, G->dscal, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
  else
    TRY(write_scalar(G, compliance, G->dscal));
  if (io.h1 || io.h2 || io.h3) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_gradient(tomo_grid* G, const T* z, double* compliance, T* dcdz, T* dvdz,
                        tomo_solve_info* info) {
  GradIO io;
  TRY(gradient_begin<T>(G, z, dcdz, dvdz, &io));
  // S3-S5: PCG from a zero start (or from the previous solution, see tomo_set_warm_start)
  tomo_status st = pcg<T>(G, G->warm_gradient && G->have_solution, info);
  if (st != TOMO_OK) return st;
  TRY(pmark(G, 3));
  return gradient_end<T>(G, io, compliance, dcdz, dvdz);
}

// Eq. 3 for the objective J = l^T u: K lambda = l (K symmetric), then
// dJ/drho_e = -p rho^(p-1) (E0-Emin) h lambda_e^T K0 u_e and dJ/dz = P^T dJ/drho.
template <typename T>
tomo_status do_adjoint(tomo_grid* G, const T* z, const T* l, double* J, T* djdz,
                       tomo_solve_info* info_u, tomo_solve_info* info_l) {
  if (!z || !l || !djdz) return fail(G, TOMO_EINVAL, "null array");
  const Geom& g = G->g;
  const int n = 3 * g.nn;
  const size_t be = sizeof(T) * (size_t)g.nel, bn = sizeof(T) * (size_t)n;
  const tomo_grid_desc& d = G->d;
  const void *dz, *dl;
  void* ddj;
  bool h1, h2, h3;
  TRY(stage_in(G, z, be, 0, &dz, &h1));
  TRY(stage_in(G, l, bn, 2, &dl, &h2));
  TRY(stage_out(G, djdz, be, 1, &ddj, &h3));
  if (!G->adj_T) {
    TRY(dalloc(G, &G->adj_T, bn));
    TRY(dalloc(G, (void**)&G->adj64, sizeof(double) * (size_t)n));
    TRY(dalloc(G, &G->adj_hi, bn));
    if (G->prec == TOMO_FP32) TRY(dalloc(G, &G->adj_lo, bn));
  }
  // the adjoint load, masked like f, and its norm (tolerance of the adjoint solve)
  CK(launch_mask_copy<T>(G->stream, g, (const T*)dl, G->L[0].mask, (T*)G->adj_T));
  CK(launch_convert<double, T>(G->stream, n, (const T*)G->adj_T, nullptr, G->adj64));
  CK(launch_dot<double, double>(G->stream, n, G->adj64, G->adj64, nullptr, G->partials,
                                G->counter, G->dscal + 2));
  G->launches += 3;
  CK(cudaMemcpyAsync(G->h_scal, G->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost,
                     G->stream));
  TRY(sync(G));
  const double lff = *G->h_scal;
  T* rho = (T*)G->rho;
  CK(launch_filter<T>(G->stream, g, G->d_taps, (const T*)G->d_tapw, G->ntaps, G->filter_radius,
                      (const T*)dz, (const T*)G->Hs, rho, 0, 1, (T)d.E0, (T)d.Emin,
                      (T)d.penal, (T)d.h, (T*)G->L[0].s));
  G->launches += 1;
  TRY(setup_levels<T>(G));
  // adjoint solve, from zero, with its own right-hand side
  G->rhs_T = G->adj_T;
  G->rhs64 = G->adj64;
  G->rhs_ff = lff;
  G->rhs_id = 1;
  tomo_status st = pcg<T>(G, false, info_l);
  G->rhs_T = G->f_T;
  G->rhs64 = G->f64;
  G->rhs_ff = G->ff;
  G->rhs_id = 0;
  if (st != TOMO_OK) return st;
  CK(cudaMemcpyAsync(G->adj_hi, G->xhi, bn, cudaMemcpyDeviceToDevice, G->stream));
  if (G->adj_lo)
    CK(cudaMemcpyAsync(G->adj_lo, G->xlo, bn, cudaMemcpyDeviceToDevice, G->stream));
  // state solve (from zero: the iterate holds lambda)
  st = pcg<T>(G, false, info_u);
  if (st != TOMO_OK) return st;
  CK(launch_dot<double, T>(G->stream, n, G->adj64, (const T*)G->xhi, (const T*)x_lo<T>(G),
                           G->partials, G->counter, G->dscal));
  CK(launch_sensitivity<T>(G->stream, g, rho, (const T*)G->xhi, (const T*)x_lo<T>(G),
                           (const T*)G->adj_hi, (const T*)G->adj_lo, elem_const<T>(G),
                           (T)d.penal, (T)d.E0, (T)d.Emin, (T)d.h, (T*)G->dcp));
  CK(launch_filter<T>(G->stream, g, G->d_taps, (const T*)G->d_tapw, G->ntaps, G->filter_radius,
                      (const T*)G->dcp, (const T*)G->Hs, (T*)ddj, 1, 0, T(0), T(0), T(0), T(0),
                      nullptr));
  G->launches += 3;
  TRY(copy_back(G, djdz, ddj, be, h3));
  TRY(write_scalar(G, J, G->dscal));
  if (h1 || h2 || h3) TRY(sync(G));
  return TOMO_OK;
}

template <typename T>
tomo_status do_get_u(tomo_grid* G, T* u) {
  if (!u) return fail(G, TOMO_EINVAL, "null array");
  if (!G->have_solution) return fail(G, TOMO_EINVAL, "no solution computed yet");
  const size_t bn = sizeof(T) * 3 * (size_t)G->g.nn;
  void* dout;
  bool hout;
  TRY(stage_out(G, u, bn, 3, &dout, &hout));
  CK(launch_convert<T, T>(G->stream, 3 * G->g.nn, (const T*)G->xhi, (const T*)x_lo<T>(G),
                          (T*)dout));
  G->launches += 1;
  TRY(copy_back(G, u, dout, bn, hout));
  if (hout) TRY(sync(G));
  return TOMO_OK;
}

// ---------------------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------------------
double lam_max_element(const double K0[576]) {
  // power iteration on diag(K0)^-1 K0 (similar to a symmetric matrix, eigenvalues >= 0)
  std::vector<double> x(24), y(24);
  for (int i = 0; i < 24; ++i) x[i] = 1.0 + 0.01 * i * ((i & 1) ? -1 : 1);
  double lam = 0.0;
  for (int it = 0; it < 2000; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < 24; ++i) {
      double s = 0.0;
      for (int j = 0; j < 24; ++j) s += K0[i * 24 + j] * x[j];
      y[i] = s / K0[i * 25];
      nrm += y[i] * y[i];
    }
    nrm = std::sqrt(nrm);
    double xn = 0.0;
    for (int i = 0; i < 24; ++i) xn += x[i] * x[i];
    lam = nrm / std::sqrt(xn);
    for (int i = 0; i < 24; ++i) x[i] = y[i] / nrm;
  }
  return lam;
}

std::vector<uint8_t> coarse_mask(const Geom& gf, const std::vector<uint8_t>& mf, const Geom& gc) {
  std::vector<uint8_t> mc(gc.nn, 0);
  for (int K = 0; K < gc.nzn; ++K)
    for (int J = 0; J < gc.nyn; ++J)
      for (int I = 0; I < gc.nxn; ++I) {
        uint8_t m = 0;
        for (int dz = -1; dz <= 1; ++dz) {
          const int k = 2 * K + dz;
          if (k < 0 || k >= gf.nzn) continue;
          for (int dy = -1; dy <= 1; ++dy) {
            const int j = 2 * J + dy;
            if (j < 0 || j >= gf.nyn) continue;
            for (int dx = -1; dx <= 1; ++dx) {
              const int i = 2 * I + dx;
              if (i < 0 || i >= gf.nxn) continue;
              m |= mf[i + gf.nxn * (j + gf.nyn * k)];
            }
          }
        }
        mc[I + gc.nxn * (J + gc.nyn * K)] = m;
      }
  return mc;
}

void free_grid(tomo_grid* G) {
  if (!G) return;
  // nothing of the grid may still run; its buffers go back to the pool in stream order
  cudaStream_t st = G->stream;
  if (G->side) cudaStreamSynchronize(G->side);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  auto F = [st](void* p) {
    if (p && cudaFreeAsync(p, st) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p);
    }
  };
  for (auto& Lv : G->L) {
    F(Lv.s);
    F(Lv.mask);
    F(Lv.b);
    F(Lv.x);
    F(Lv.xp);
    F(Lv.t);
    F(Lv.tile_fixed);
    F(Lv.invd);
  }
  F(G->d_taps);
  F(G->d_tapw);
  F(G->Hs);
  F(G->dvdz);
  F(G->coarseA);
  F(G->coarseD);
  F(G->f_T);
  F(G->f64);
  F(G->r);
  F(G->p);
  F(G->q);
  F(G->xhi);
  F(G->xlo);
  F(G->rho);
  F(G->dcp);
  F(G->s64);
  F(G->partials);
  F(G->counter);
  F(G->vt_eb);
  F(G->sc);
  F(G->dscal);
  pinned_put(G->h_sc);
  pinned_put(G->h_scal);
  for (void* s : G->stage) F(s);
  if (G->loop_exec) cudaGraphExecDestroy(G->loop_exec);
  if (G->loop_exec_adj) cudaGraphExecDestroy(G->loop_exec_adj);
  for (auto& e : G->loop_cache) cudaGraphExecDestroy(e.exec);
  G->loop_cache.clear();
  F(G->load_idx);
  F(G->load_val);
  G->invd = nullptr;  // (level 0's D^-1, freed with the levels)
  F(G->adj_T);
  F(G->adj64);
  F(G->adj_hi);
  F(G->adj_lo);
  if (G->cap_stream) cudaStreamDestroy(G->cap_stream);
  if (G->side) cudaStreamDestroy(G->side);
  if (G->ev_fork) cudaEventDestroy(G->ev_fork);
  if (G->ev_factor) cudaEventDestroy(G->ev_factor);
  for (auto e : G->ev) cudaEventDestroy(e);
  for (auto e : G->phase_ev)
    if (e) cudaEventDestroy(e);
  if (tomo::g_cur_err == &G->err) tomo::g_cur_err = nullptr;
  delete G;
}

// Multigrid level grids: ceil-halving until the coarsest has 3 N_n <= 192 (or mg_levels
// levels, when set, with a coarsest of at most kMaxDenseDofs), at least two levels.
std::vector<Geom> plan_levels(const tomo_grid_desc& d) {
  std::vector<Geom> v{make_geom(d.nx, d.ny, d.nz)};
  if (d.precond != TOMO_PRECOND_MG) return v;
  const int want = d.mg_levels;
  while (true) {
    const Geom gf = v.back();
    const int nl = (int)v.size();
    const bool small = 3 * gf.nn <= 192;
    const bool can = std::max(gf.nx, std::max(gf.ny, gf.nz)) > 1;
    if (!can) break;
    if (want > 0 && nl >= want && 3 * gf.nn <= kMaxDenseDofs) break;
    if (want <= 0 && small) break;
    v.push_back(make_geom((gf.nx + 1) / 2, (gf.ny + 1) / 2, (gf.nz + 1) / 2));
  }
  if (v.size() < 2) {
    // a single-level grid: the dense solve of the grid itself would be the whole solve;
    // keep one coarse level so that the V-cycle structure holds
    const Geom gf = v.back();
    v.push_back(make_geom((gf.nx + 1) / 2, (gf.ny + 1) / 2, (gf.nz + 1) / 2));
  }
  return v;
}

// Upper estimate of the device bytes a grid with this descriptor allocates, host staging
// of z, dc/dz and dV/dz included (the allocations of create_impl plus 25 % and 4 MiB for
// allocation granularity and the captured CG loop).
size_t estimate_device_bytes(const tomo_grid_desc& d) {
  const size_t T = d.precision == TOMO_FP64 ? 8 : 4;
  const std::vector<Geom> lv = plan_levels(d);
  const Geom& g = lv[0];
  size_t b = 0;
  for (size_t l = 0; l < lv.size(); ++l) {
    const size_t nv = 3 * (size_t)lv[l].nn * T;
    b += (size_t)lv[l].nel * T + (size_t)lv[l].nn + (l > 0 ? 4 : 3) * nv;
  }
  if (d.precond == TOMO_PRECOND_MG) {
    const size_t nc = 3 * (size_t)lv.back().nn;
    b += nc * nc * T + nc * T;
    if (d.precision == TOMO_FP32)  // D^-1 per node on the smoothed levels
      for (size_t l = 0; l + 1 < lv.size(); ++l) b += (size_t)lv[l].nn * T;
  }
  const size_t nv = 3 * (size_t)g.nn * T, ne = (size_t)g.nel * T;
  b += nv + 3 * (size_t)g.nn * 8 + 4 * nv + 4 * ne + 3 * ne;
  if (d.precision == TOMO_FP32) b += nv + (size_t)g.nel * 8;
  b += sizeof(double) * (size_t)std::max(1 << 16, oc_partials_needed(g.nel));
  return b + b / 4 + (4u << 20);
}

template <typename T>
tomo_status create_impl(tomo_grid* G) {
  const Geom g = G->g;
  const size_t nv = sizeof(T) * 3 * (size_t)g.nn, ne = sizeof(T) * (size_t)g.nel;
  // levels
  {
    tomo_level L0;
    L0.g = g;
    L0.h = G->d.h;
    L0.hmask.assign(g.nn, 0);
    for (int c = 0; c < 3; ++c)
      for (int n = 0; n < g.nn; ++n)
        if (G->fixed[(size_t)c * g.nn + n]) L0.hmask[n] |= (uint8_t)(1u << c);
    G->L.push_back(std::move(L0));
  }
  if (G->d.precond == TOMO_PRECOND_MG) {
    const std::vector<Geom> dims = plan_levels(G->d);
    for (size_t l = 1; l < dims.size(); ++l) {
      tomo_level Lc;
      Lc.g = dims[l];
      Lc.h = G->L.back().h * 2.0;
      Lc.hmask = coarse_mask(G->L.back().g, G->L.back().hmask, Lc.g);
      G->L.push_back(std::move(Lc));
    }
    G->coarse_n = 3 * G->L.back().g.nn;
    if (G->coarse_n > kMaxDenseDofs)
      return fail(G, TOMO_EINVAL, "coarsest level has %d DOFs (> %d); use more levels",
                  G->coarse_n, kMaxDenseDofs);
  }
  for (size_t l = 0; l < G->L.size(); ++l) {
    auto& Lv = G->L[l];
    const size_t lnv = sizeof(T) * 3 * (size_t)Lv.g.nn;
    TRY(dalloc(G, &Lv.s, sizeof(T) * (size_t)Lv.g.nel));
    TRY(dalloc(G, (void**)&Lv.mask, Lv.g.nn));
    CK(cudaMemcpyAsync(Lv.mask, Lv.hmask.data(), Lv.g.nn, cudaMemcpyHostToDevice, G->stream));
    if (l > 0) TRY(dalloc(G, &Lv.b, lnv));
    TRY(dalloc(G, &Lv.x, lnv));
    TRY(dalloc(G, &Lv.xp, lnv));
    TRY(dalloc(G, &Lv.t, lnv));
    if (sizeof(T) == 4) {
      const std::vector<uint8_t> fl = march2_tile_flags(Lv.g, Lv.hmask);
      TRY(dalloc(G, (void**)&Lv.tile_fixed, fl.size()));
      CK(cudaMemcpyAsync(Lv.tile_fixed, fl.data(), fl.size(), cudaMemcpyHostToDevice,
                         G->stream));
    }
  }
  if (G->coarse_n > 0 && sizeof(T) == 4) {
    // D^-1 per node on every smoothed level (the Chebyshev steps of k_march2 read it; the
    // finest one also serves the zero-start step fused into the CG update)
    for (size_t l = 0; l + 1 < G->L.size(); ++l)
      TRY(dalloc(G, &G->L[l].invd, sizeof(T) * (size_t)G->L[l].g.nn));
    G->invd = G->L[0].invd;
    G->fuse_j0 = true;
    // the coarse tail in one cluster launch: from the first level (below the finest and
    // above the coarsest) with few enough elements for the cluster's threads
    const int nl = (int)G->L.size();
    for (int l = 1; l + 1 < nl; ++l)
      if (G->L[l].g.nel <= kVtMaxTailElements && nl - l <= kVtMaxLevels && vtail_ctas() > 0) {
        G->vt_level = l;
        G->vt_ld = G->L[l].g.nel;
        TRY(dalloc(G, &G->vt_eb, sizeof(float) * 24 * (size_t)G->vt_ld));
        break;
      }
  }
  if (G->coarse_n > 0) {
    TRY(dalloc(G, &G->coarseA, sizeof(T) * (size_t)G->coarse_n * G->coarse_n));
    TRY(dalloc(G, &G->coarseD, sizeof(T) * (size_t)G->coarse_n));
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&G->side, cudaStreamNonBlocking, greatest));
    CK(cudaEventCreateWithFlags(&G->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&G->ev_factor, cudaEventDisableTiming));
  }
  // fine vectors
  TRY(dalloc(G, &G->f_T, nv));
  TRY(dalloc(G, (void**)&G->f64, sizeof(double) * 3 * (size_t)g.nn));
  TRY(dalloc(G, &G->r, nv));
  TRY(dalloc(G, &G->p, nv));
  TRY(dalloc(G, &G->q, nv));
  TRY(dalloc(G, &G->xhi, nv));
  if (G->prec == TOMO_FP32) TRY(dalloc(G, &G->xlo, nv));
  if (G->prec == TOMO_FP32 && G->d.rr_every > 0) {
    TRY(dalloc(G, (void**)&G->s64, sizeof(double) * (size_t)g.nel));
  }
  TRY(dalloc(G, &G->rho, ne));
  TRY(dalloc(G, &G->dcp, ne));
  TRY(dalloc(G, &G->Hs, ne));
  TRY(dalloc(G, &G->dvdz, ne));
  {
    // the load is sparse (point, line or face loads): zero both copies on the device and
    // scatter the nonzero free entries
    std::vector<int64_t> idx;
    std::vector<double> val;
    G->ff = 0.0;
    for (size_t k = 0; k < G->f.size(); ++k)
      if (!G->fixed[k] && G->f[k] != 0.0) {
        idx.push_back((int64_t)k);
        val.push_back(G->f[k]);
        G->ff += G->f[k] * G->f[k];
      }
    CK(cudaMemsetAsync(G->f_T, 0, nv, G->stream));
    CK(cudaMemsetAsync(G->f64, 0, sizeof(double) * 3 * (size_t)g.nn, G->stream));
    if (!idx.empty()) {  // kept: the compliance f^T u and the CG start use the entries
      G->load_nnz = (int)idx.size();
      TRY(dalloc(G, (void**)&G->load_idx, sizeof(int64_t) * idx.size()));
      TRY(dalloc(G, (void**)&G->load_val, sizeof(double) * val.size()));
      CK(cudaMemcpyAsync(G->load_idx, idx.data(), sizeof(int64_t) * idx.size(),
                         cudaMemcpyHostToDevice, G->stream));
      CK(cudaMemcpyAsync(G->load_val, val.data(), sizeof(double) * val.size(),
                         cudaMemcpyHostToDevice, G->stream));
      CK(launch_scatter_load<T>(G->stream, G->load_nnz, G->load_idx, G->load_val, (T*)G->f_T,
                                G->f64));
      G->launches += 1;
    }
  }
  G->rhs_T = G->f_T;
  G->rhs64 = G->f64;
  G->rhs_ff = G->ff;
  G->rhs_id = 0;
  // reductions
  G->partials_n = std::max(1 << 16, oc_partials_needed(g.nel));
  TRY(dalloc(G, (void**)&G->partials, sizeof(double) * (size_t)G->partials_n));
  TRY(dalloc(G, (void**)&G->counter, sizeof(unsigned) * 4));
  CK(cudaMemsetAsync(G->counter, 0, sizeof(unsigned) * 4, G->stream));
  TRY(dalloc(G, (void**)&G->sc, sizeof(CgScalars)));
  CK(cudaMemsetAsync(G->sc, 0, sizeof(CgScalars), G->stream));
  TRY(dalloc(G, (void**)&G->dscal, sizeof(double) * 8));
  G->h_sc = static_cast<CgScalars*>(pinned_get(sizeof(CgScalars)));
  G->h_scal = static_cast<double*>(pinned_get(sizeof(double) * 8));
  if (!G->h_sc || !G->h_scal) return fail(G, TOMO_ENOMEM, "pinned host memory");
  // filter taps and weight sums
  G->taps = filter_taps(G->d.rmin);
  G->ntaps = (int)G->taps.size();
  G->filter_radius = 0;
  for (const auto& t : G->taps)
    G->filter_radius = std::max(G->filter_radius,
                                std::max(std::abs(t.di), std::max(std::abs(t.dj), std::abs(t.dk))));
  {
    std::vector<int4> t4(G->ntaps);
    std::vector<T> tw(G->ntaps);
    for (int q = 0; q < G->ntaps; ++q) {
      t4[q] = make_int4(G->taps[q].di, G->taps[q].dj, G->taps[q].dk, 0);
      tw[q] = (T)G->taps[q].w;
    }
    TRY(dalloc(G, (void**)&G->d_taps, sizeof(int4) * std::max(1, G->ntaps)));
    TRY(dalloc(G, &G->d_tapw, sizeof(T) * std::max(1, G->ntaps)));
    CK(cudaMemcpyAsync(G->d_taps, t4.data(), sizeof(int4) * G->ntaps, cudaMemcpyHostToDevice,
                       G->stream));
    CK(cudaMemcpyAsync(G->d_tapw, tw.data(), sizeof(T) * G->ntaps, cudaMemcpyHostToDevice,
                       G->stream));
    CK(launch_fill<T>(G->stream, g.nel, (T*)G->dcp, T(1)));
    CK(launch_filter<T>(G->stream, g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                        G->filter_radius,
                        (const T*)G->dcp, nullptr, (T*)G->Hs, 2, 0, T(0), T(0), T(0), T(0),
                        nullptr));
    G->launches += 1;
    TRY(sync(G));
  }
  return TOMO_OK;
}

// Chebyshev degrees (finest level, coarser levels) and interval ratio of a grid; the
// captured CG loops, which bake them in, are dropped and rebuilt at the next solve.
// wlevels < 0 keeps the grid's cycle shape
tomo_status set_smoother(tomo_grid* G, int fine, int coarse, double ratio, double lam,
                         int64_t wlevels) {
  const uint32_t w = wlevels < 0 ? G->wlevels : (uint32_t)wlevels;
  if (fine < 1 || fine > 16 || coarse < 1 || coarse > 16 || !(ratio > 1.0) || !std::isfinite(ratio))
    return fail(G, TOMO_EINVAL, "smoother: degrees in 1..16 and ratio > 1 (got %d, %d, %g)",
                fine, coarse, ratio);
  if (std::isnan(lam))
    return fail(G, TOMO_EINVAL, "smoother bound: NaN");
  if (!(lam > 0.0)) lam = G->lam_bound;
  if (!(lam >= 0.25 * G->lam_bound && lam <= G->lam_bound))
    return fail(G, TOMO_EINVAL, "smoother bound %g outside [%g, %g] (a quarter of the element "
                "bound up to the bound)", lam, 0.25 * G->lam_bound, G->lam_bound);
  if (fine == G->d.smoother_degree && coarse == G->d.coarse_degree && ratio == G->cheb_ratio &&
      lam == G->lam_hi && w == G->wlevels)
    return TOMO_OK;
  TRY(sync(G));  // no captured loop of this grid is still running
  // keep the current load-slot loop for a later return to these settings (up to 8)
  if (G->loop_exec) {
    if (G->loop_cache.size() >= 8) {
      cudaGraphExecDestroy(G->loop_cache.front().exec);
      G->loop_cache.erase(G->loop_cache.begin());
    }
    G->loop_cache.push_back(tomo_grid::CachedLoop{G->d.smoother_degree, G->d.coarse_degree,
                                                  G->cheb_ratio, G->lam_hi, G->wlevels,
                                                  G->loop_exec});
  }
  G->loop_exec = nullptr;
  if (G->loop_exec_adj) cudaGraphExecDestroy(G->loop_exec_adj);
  G->loop_exec_adj = nullptr;
  G->d.smoother_degree = fine;
  G->d.coarse_degree = coarse;
  G->d.cheb_ratio = ratio;
  G->cheb_ratio = ratio;
  G->lam_hi = lam;
  G->wlevels = w;
  for (size_t k = 0; k < G->loop_cache.size(); ++k) {
    const tomo_grid::CachedLoop& e = G->loop_cache[k];
    if (e.fine == fine && e.coarse == coarse && e.ratio == ratio && e.lam == lam &&
        e.wlevels == w) {
      G->loop_exec = e.exec;
      G->loop_cache.erase(G->loop_cache.begin() + k);
      break;
    }
  }
  G->gen += 1;
  return TOMO_OK;
}

// The smoother autotuner: the state solve K(P z) u = f (cold start) timed with CUDA events
// on the grid's stream for each candidate setting, on each of the nz designs (one untimed
// solve, which also captures the candidate's loop unless the grid kept it, then the median
// of reps), the medians summed over the designs; the fastest candidate that converges on
// every design is kept.
template <typename T>
tomo_status do_autotune(tomo_grid* G, const T* const* zs, int nz, const int32_t* pairs, int n,
                        int reps, tomo_tune_result* res, int32_t* best) {
  // (fine, coarse) degrees: (2, 2) is fastest on random fields, (1, 4) on OC-evolved
  // designs (near 0/1 densities), measured on the 192x96x76 MBB-type block; with the
  // built-in list each pair is also tried at 0.75 and 0.68 of the element bound of the
  // smoothing interval (lambda_max of D^-1 K is near 3.1-3.9 on those designs, well below
  // the bound of 5.3, which only isolated elements reach)
  static const int32_t kDefault[] = {2, 2, 2, 3, 2, 4, 1, 3, 1, 4, 1, 6};
  static const double kBoundScale[] = {1.0, 0.75, 0.68};
  // after the V-cycle candidates of the built-in list, the best of them is tried with a
  // W-cycle at level 1 and at levels 1 and 2 (bit masks 2 and 6); then the best so far with
  // the interval [lam/ratio, lam] at ratios 12, 30 and 50 instead of the grid's
  static const uint32_t kWStage[] = {2u, 6u};
  static const double kRatioStage[] = {12.0, 30.0, 50.0};
  if (!zs || nz < 1 || nz > 16) return fail(G, TOMO_EINVAL, "autotune: 1..16 designs");
  for (int d = 0; d < nz; ++d)
    if (!zs[d]) return fail(G, TOMO_EINVAL, "null array");
  struct Cand {
    int fine, coarse;
    double lam, ratio;
    uint32_t w;
  };
  const double ratio0 = G->cheb_ratio;
  std::vector<Cand> cands;
  std::vector<int> stage_end;  // candidates [stage_end[s-1], stage_end[s]) form stage s
  if (!pairs) {
    for (double f : kBoundScale)
      for (size_t k = 0; k + 1 < sizeof(kDefault) / sizeof(kDefault[0]); k += 2)
        cands.push_back(Cand{kDefault[k], kDefault[k + 1], f * G->lam_bound, ratio0, 0u});
    const int nv = (int)cands.size();
    stage_end = {nv, nv + 2, nv + 5};
  } else {
    if (n < 1 || n > 64)
      return fail(G, TOMO_EINVAL, "autotune: 1..64 candidates and 1..16 repetitions");
    for (int k = 0; k < n; ++k)
      cands.push_back(Cand{pairs[2 * k], pairs[2 * k + 1], G->lam_hi, ratio0, G->wlevels});
    stage_end = {n};
  }
  const int ntot = stage_end.back();
  if (reps < 1 || reps > 16)
    return fail(G, TOMO_EINVAL, "autotune: 1..64 candidates and 1..16 repetitions");
  if (G->d.precond != TOMO_PRECOND_MG)
    return fail(G, TOMO_EINVAL, "autotune: the grid has no multigrid smoother");
  for (int k = 0; k < stage_end[0]; ++k)
    if (cands[k].fine < 1 || cands[k].fine > 16 || cands[k].coarse < 1 || cands[k].coarse > 16)
      return fail(G, TOMO_EINVAL, "autotune: candidate %d has a degree outside 1..16", k);
  const int fine0 = G->d.smoother_degree, coarse0 = G->d.coarse_degree;
  const double lam0 = G->lam_hi;
  const uint32_t w0 = G->wlevels;
  const size_t be = sizeof(T) * (size_t)G->g.nel;
  const tomo_grid_desc& d = G->d;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    CK(cudaGetLastError());
  }
  std::vector<double> sum(ntot, 0.0);
  std::vector<int> iters(ntot, 0), status(ntot, TOMO_OK);
  int bi = -1;
  tomo_status st = TOMO_OK;
  int k0 = 0;
  for (size_t sg = 0; sg < stage_end.size() && st == TOMO_OK; ++sg) {
    if (sg > 0) {  // the next stage starts from the best candidate so far
      if (bi < 0) break;
      const Cand b = cands[bi];
      if (sg == 1)
        for (uint32_t w : kWStage) cands.push_back(Cand{b.fine, b.coarse, b.lam, b.ratio, w});
      else
        for (double r : kRatioStage) cands.push_back(Cand{b.fine, b.coarse, b.lam, r, b.w});
    }
    const int k1 = stage_end[sg];
    for (int dsg = 0; dsg < nz && st == TOMO_OK; ++dsg) {
      // the material of design dsg
      const void* dz;
      bool h1;
      st = stage_in(G, zs[dsg], be, 0, &dz, &h1);
      if (st != TOMO_OK) break;
      if (launch_filter<T>(G->stream, G->g, G->d_taps, (const T*)G->d_tapw, G->ntaps,
                           G->filter_radius, (const T*)dz, (const T*)G->Hs, (T*)G->rho, 0, 1,
                           (T)d.E0, (T)d.Emin, (T)d.penal, (T)d.h, (T*)G->L[0].s) !=
          cudaSuccess) {
        cudaGetLastError();
        st = fail(G, TOMO_ECUDA, "autotune: filter launch failed");
        break;
      }
      G->launches += 1;
      st = setup_levels<T>(G);
      if (st != TOMO_OK) break;
      for (int k = k0; k < k1 && st == TOMO_OK; ++k) {
        if (status[k] != TOMO_OK) continue;  // failed on an earlier design
        st = set_smoother(G, cands[k].fine, cands[k].coarse, cands[k].ratio, cands[k].lam,
                          cands[k].w);
        if (st != TOMO_OK) break;
        tomo_solve_info info{};
        // untimed solve, which captures this candidate's loop, unless the grid kept it; a
        // candidate is timed as it is, without the fallback to the element bound
        tomo_status sk = TOMO_OK;
        if (!G->loop_exec || G->prof) sk = pcg<T>(G, false, &info, false);
        std::vector<double> ms;
        for (int r = 0; r < reps && sk == TOMO_OK; ++r) {
          float t = 0.0f;
          if (cudaEventRecord(e0, G->stream) != cudaSuccess) sk = TOMO_ECUDA;
          if (sk == TOMO_OK) sk = pcg<T>(G, false, &info, false);
          if (sk == TOMO_OK && (cudaEventRecord(e1, G->stream) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            sk = TOMO_ECUDA;
          ms.push_back(t);
        }
        if (sk == TOMO_ECUDA) {
          cudaGetLastError();
          st = fail(G, TOMO_ECUDA, "autotune: CUDA error while timing candidate %d", k);
          break;
        }
        status[k] = sk;
        iters[k] = std::max(iters[k], (int)info.iters);
        if (sk == TOMO_OK) {
          std::sort(ms.begin(), ms.end());
          sum[k] += ms[ms.size() / 2];
        }
      }
    }
    for (int k = k0; k < k1; ++k)
      if (status[k] == TOMO_OK && (bi < 0 || sum[k] < sum[bi])) bi = k;
    k0 = k1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (res)
    for (int k = 0; k < ntot; ++k) {
      const bool ran = k < (int)cands.size();
      res[k].fine_degree = ran ? cands[k].fine : 0;
      res[k].coarse_degree = ran ? cands[k].coarse : 0;
      res[k].iters = iters[k];
      res[k].status = ran ? status[k] : TOMO_ENOCONV;
      res[k].ms = (ran && status[k] == TOMO_OK && k < k0) ? sum[k] : -1.0;
      res[k].lam = ran ? cands[k].lam : 0.0;
      res[k].w_levels = ran ? cands[k].w : 0u;
      res[k].reserved = 0u;
      res[k].ratio = ran ? cands[k].ratio : 0.0;
    }
  if (st == TOMO_OK && bi < 0)
    st = fail(G, TOMO_ENOCONV, "autotune: no candidate converged");
  if (st != TOMO_OK) {
    std::string why = G->err;
    set_smoother(G, fine0, coarse0, ratio0, lam0, w0);
    G->err = why;
    return st;
  }
  TRY(set_smoother(G, cands[bi].fine, cands[bi].coarse, cands[bi].ratio, cands[bi].lam,
                   cands[bi].w));
  if (best) *best = bi;
  return TOMO_OK;
}

}  // namespace

// =======================================================================================
// extern "C"
// =======================================================================================
extern "C" {

void tomo_default_desc(tomo_grid_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->nx = d->ny = d->nz = 1;
  d->h = 1.0;
  d->E0 = 1.0;
  d->Emin = 1e-9;
  d->nu = 0.3;
  d->penal = 3.0;
  d->rmin = 1.5;
  d->precision = TOMO_FP32;
  d->precond = TOMO_PRECOND_MG;
  d->rtol = 1e-6;
  d->maxit = 2000;
  d->mg_levels = 0;
  d->smoother_degree = 2;
  d->coarse_degree = 0;
  d->cheb_ratio = 20.0;
  d->cheb_lmax = 0.0;
  d->rr_every = 50;
  d->stream = nullptr;
}

tomo_status tomo_create_grid(const tomo_grid_desc* desc, tomo_grid** out) {
  tomo_grid* G = nullptr;
  if (!desc || !out) return fail(nullptr, TOMO_EINVAL, "null descriptor or output");
  *out = nullptr;
  const tomo_grid_desc& d = *desc;
  if (d.nx < 1 || d.ny < 1 || d.nz < 1)
    return fail(nullptr, TOMO_EINVAL, "grid dimensions must be >= 1 (got %d %d %d)", d.nx, d.ny,
                d.nz);
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  if (3 * nn >= (1LL << 31) - 1)
    return fail(nullptr, TOMO_EINVAL, "grid too large for 32-bit nodal indexing");
  if (!(d.h > 0.0) || !(d.E0 > d.Emin) || !(d.Emin >= 0.0) || !(d.nu > -1.0 && d.nu < 0.5) ||
      !(d.penal >= 1.0) || !(d.rmin > 0.0) || d.rmin > 16.0)
    return fail(nullptr, TOMO_EINVAL,
                "invalid material/filter parameters (need h>0, E0>Emin>=0, -1<nu<0.5, p>=1, "
                "0<rmin<=16)");
  if (!d.fixed_dof || !d.f) return fail(nullptr, TOMO_EINVAL, "fixed_dof and f are required");
  if (d.precision != TOMO_FP64 && d.precision != TOMO_FP32)
    return fail(nullptr, TOMO_EINVAL, "unknown precision %d", d.precision);
  if (d.precond != TOMO_PRECOND_MG && d.precond != TOMO_PRECOND_JACOBI)
    return fail(nullptr, TOMO_EINVAL, "unknown preconditioner %d", d.precond);
  G = new (std::nothrow) tomo_grid();
  if (!G) return fail(nullptr, TOMO_ENOMEM, "host allocation failed");
  G->d = d;
  G->d.fixed_dof = nullptr;
  G->d.f = nullptr;
  if (G->d.rtol <= 0.0) G->d.rtol = 1e-6;
  if (G->d.maxit <= 0) G->d.maxit = 2000;
  if (G->d.smoother_degree <= 0) G->d.smoother_degree = 2;
  if (G->d.coarse_degree <= 0) G->d.coarse_degree = G->d.smoother_degree;
  if (G->d.rr_every == 0) G->d.rr_every = 50;
  G->cheb_ratio = G->d.cheb_ratio > 1.0 ? G->d.cheb_ratio : 20.0;
  G->prec = d.precision;
  G->tsize = d.precision == TOMO_FP64 ? 8 : 4;
  G->stream = (cudaStream_t)d.stream;
  G->g = make_geom(d.nx, d.ny, d.nz);
  G->fixed.assign(d.fixed_dof, d.fixed_dof + 3 * nn);
  for (auto& v : G->fixed) v = v ? 1 : 0;
  G->f.assign(d.f, d.f + 3 * nn);
  g_cur_err = &G->err;
  if (cudaGetDevice(&G->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&G->num_sms, cudaDevAttrMultiProcessorCount, G->device) !=
          cudaSuccess) {
    cudaGetLastError();
    tomo::g_cur_err = nullptr;
    delete G;
    return fail(nullptr, TOMO_ECUDA, "no usable CUDA device");
  }
  build_unit_stiffness(d.nu, G->K0);
  if (!build_hadamard_blocks(G->K0, G->blk, &G->k0diag)) {
    tomo::g_cur_err = nullptr;
    delete G;
    return fail(nullptr, TOMO_EINVAL, "element stiffness is not cube-symmetric");
  }
  if (!block_kinds(G->blk, &G->kinds)) {
    tomo::g_cur_err = nullptr;
    delete G;
    return fail(nullptr, TOMO_EINVAL, "element stiffness blocks are not of the isotropic kinds");
  }
  G->lam_bound = lam_max_element(G->K0);
  G->lam_hi = G->d.cheb_lmax > 0.0 ? G->d.cheb_lmax : G->lam_bound;
  tomo_status st = G->prec == TOMO_FP64 ? create_impl<double>(G) : create_impl<float>(G);
  if (st != TOMO_OK) {
    g_create_err = G->err;
    free_grid(G);
    return st;
  }
  *out = G;
  return TOMO_OK;
}

tomo_status tomo_destroy_grid(tomo_grid* G) {
  if (!G) return TOMO_OK;
  cudaStreamSynchronize(G->stream);
  free_grid(G);
  return TOMO_OK;
}

tomo_status tomo_grid_device_bytes(const tomo_grid* G, size_t* bytes) {
  if (!G || !bytes) return TOMO_EINVAL;
  *bytes = G->dev_bytes;
  return TOMO_OK;
}

tomo_status tomo_estimate_device_bytes(const tomo_grid_desc* d, size_t* bytes) {
  if (!d || !bytes || d->nx < 1 || d->ny < 1 || d->nz < 1) return TOMO_EINVAL;
  *bytes = estimate_device_bytes(*d);
  return TOMO_OK;
}

tomo_status tomo_set_warm_start(tomo_grid* G, int32_t on) {
  if (!G) return TOMO_EINVAL;
  G->warm_gradient = on != 0;
  return TOMO_OK;
}

tomo_status tomo_set_smoother(tomo_grid* G, int32_t fine_degree, int32_t coarse_degree,
                              double ratio) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  return set_smoother(G, fine_degree, coarse_degree, ratio, G->lam_hi);
}
tomo_status tomo_set_smoother_bound(tomo_grid* G, double lam) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  if (G->d.precond != TOMO_PRECOND_MG)
    return fail(G, TOMO_EINVAL, "smoother bound: the grid has no multigrid smoother");
  return set_smoother(G, G->d.smoother_degree, G->d.coarse_degree, G->cheb_ratio, lam);
}
tomo_status tomo_get_smoother_bound(const tomo_grid* G, double* lam, double* element_bound,
                                    int64_t* fallbacks) {
  if (!G) return TOMO_EINVAL;
  if (lam) *lam = G->lam_hi;
  if (element_bound) *element_bound = G->lam_bound;
  if (fallbacks) *fallbacks = G->bound_fallbacks;
  return TOMO_OK;
}

tomo_status tomo_get_smoother(const tomo_grid* G, int32_t* fine_degree, int32_t* coarse_degree,
                              double* ratio) {
  if (!G) return TOMO_EINVAL;
  if (fine_degree) *fine_degree = G->d.smoother_degree;
  if (coarse_degree) *coarse_degree = G->d.coarse_degree;
  if (ratio) *ratio = G->cheb_ratio;
  return TOMO_OK;
}

tomo_status tomo_autotune_smoother(tomo_grid* G, const float* z, const int32_t* pairs,
                                   int32_t n, int32_t reps, tomo_tune_result* results,
                                   int32_t* best) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  TRY(check_prec(G, false));
  const float* zs[1] = {z};
  return do_autotune<float>(G, zs, 1, pairs, n, reps, results, best);
}

tomo_status tomo_autotune_smoother_d(tomo_grid* G, const double* z, const int32_t* pairs,
                                     int32_t n, int32_t reps, tomo_tune_result* results,
                                     int32_t* best) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  TRY(check_prec(G, true));
  const double* zs[1] = {z};
  return do_autotune<double>(G, zs, 1, pairs, n, reps, results, best);
}

tomo_status tomo_autotune_smoother_multi(tomo_grid* G, const float* const* z, int32_t nz,
                                         const int32_t* pairs, int32_t n, int32_t reps,
                                         tomo_tune_result* results, int32_t* best) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  TRY(check_prec(G, false));
  return do_autotune<float>(G, z, nz, pairs, n, reps, results, best);
}

tomo_status tomo_autotune_smoother_multi_d(tomo_grid* G, const double* const* z, int32_t nz,
                                           const int32_t* pairs, int32_t n, int32_t reps,
                                           tomo_tune_result* results, int32_t* best) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  TRY(check_prec(G, true));
  return do_autotune<double>(G, z, nz, pairs, n, reps, results, best);
}

tomo_status tomo_set_coarse_tail(tomo_grid* G, int32_t on) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  G->err.clear();
  const bool want = on != 0 && G->vt_level > 0;
  if (want == G->vt_on) return TOMO_OK;
  TRY(sync(G));  // no captured loop of this grid is still running
  // the captured loops hold the other V-cycle form: drop them all
  if (G->loop_exec) cudaGraphExecDestroy(G->loop_exec);
  if (G->loop_exec_adj) cudaGraphExecDestroy(G->loop_exec_adj);
  G->loop_exec = G->loop_exec_adj = nullptr;
  for (auto& e : G->loop_cache) cudaGraphExecDestroy(e.exec);
  G->loop_cache.clear();
  G->vt_on = want;
  G->gen += 1;
  return TOMO_OK;
}

tomo_status tomo_get_coarse_tail(const tomo_grid* G, int32_t* level) {
  if (!G || !level) return TOMO_EINVAL;
  *level = G->vt_on ? G->vt_level : 0;
  return TOMO_OK;
}

tomo_status tomo_set_cycle(tomo_grid* G, uint32_t w_levels) {
  if (!G) return TOMO_EINVAL;
  g_cur_err = &G->err;
  G->err.clear();
  if (G->d.precond != TOMO_PRECOND_MG && w_levels != 0)
    return fail(G, TOMO_EINVAL, "cycle: the grid has no multigrid preconditioner");
  return set_smoother(G, G->d.smoother_degree, G->d.coarse_degree, G->cheb_ratio, G->lam_hi,
                      (int64_t)w_levels);
}

tomo_status tomo_get_cycle(const tomo_grid* G, uint32_t* w_levels) {
  if (!G || !w_levels) return TOMO_EINVAL;
  *w_levels = G->wlevels;
  return TOMO_OK;
}

tomo_status tomo_check_report(int32_t* checked, uint64_t* word) {
  if (!checked || !word) return TOMO_EINVAL;
  *word = 0;
#ifdef TOMO_CHECKED
  *checked = 1;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return TOMO_ECUDA;
  }
  unsigned long long (*const words[])() = {check_word_matvec2, check_word_matvec,
                                           check_word_vec, check_word_filt, check_word_vtail};
  for (auto f : words) {
    const unsigned long long w = f();
    if (w == ~0ull) return TOMO_ECUDA;
    if (*word == 0 && w != 0) *word = w;
  }
#else
  *checked = 0;
#endif
  return TOMO_OK;
}

tomo_status tomo_inject_fault(const char* site, int32_t nth) {
  if (!site || nth < 0) return TOMO_EINVAL;
  const int k = fault_site(site, std::strlen(site));
  if (k < 0) return TOMO_EINVAL;
  fault_env_once();
  g_fault_left[k].store(nth);
  return TOMO_OK;
}

tomo_status tomo_set_stream(tomo_grid* G, void* stream) {
  if (!G) return TOMO_EINVAL;
  G->stream = (cudaStream_t)stream;
  G->d.stream = stream;
  return TOMO_OK;
}

#define ENTER(G, want64)                  \
  do {                                    \
    if (!(G)) return TOMO_EINVAL;         \
    TRY(check_prec(G, want64));           \
    (G)->err.clear();                     \
    g_cur_err = &(G)->err;                \
  } while (0)

tomo_status tomo_filter(tomo_grid* G, const float* in, float* out, int transpose) {
  ENTER(G, false);
  return do_filter<float>(G, in, out, transpose);
}
tomo_status tomo_filter_d(tomo_grid* G, const double* in, double* out, int transpose) {
  ENTER(G, true);
  return do_filter<double>(G, in, out, transpose);
}
tomo_status tomo_adjoint_gradient(tomo_grid* G, const float* z, const float* l, double* J,
                                  float* djdz, tomo_solve_info* info_u,
                                  tomo_solve_info* info_l) {
  ENTER(G, false);
  return do_adjoint<float>(G, z, l, J, djdz, info_u, info_l);
}
tomo_status tomo_adjoint_gradient_d(tomo_grid* G, const double* z, const double* l, double* J,
                                    double* djdz, tomo_solve_info* info_u,
                                    tomo_solve_info* info_l) {
  ENTER(G, true);
  return do_adjoint<double>(G, z, l, J, djdz, info_u, info_l);
}
tomo_status tomo_coarse_grain(tomo_grid* G, const float* z, int32_t block, float* z_coarse) {
  ENTER(G, false);
  return do_coarse_grain<float>(G, z, block, z_coarse);
}
tomo_status tomo_coarse_grain_d(tomo_grid* G, const double* z, int32_t block,
                                double* z_coarse) {
  ENTER(G, true);
  return do_coarse_grain<double>(G, z, block, z_coarse);
}
tomo_status tomo_apply_stiffness(tomo_grid* G, const float* rho, const float* x, float* y) {
  ENTER(G, false);
  return do_apply<float>(G, rho, x, y);
}
tomo_status tomo_apply_stiffness_d(tomo_grid* G, const double* rho, const double* x, double* y) {
  ENTER(G, true);
  return do_apply<double>(G, rho, x, y);
}
tomo_status tomo_residual(tomo_grid* G, const float* rho, const float* u, const float* u_lo,
                          float* r) {
  ENTER(G, false);
  return do_residual<float>(G, rho, u, u_lo, r);
}
tomo_status tomo_residual_d(tomo_grid* G, const double* rho, const double* u, double* r) {
  ENTER(G, true);
  return do_residual<double>(G, rho, u, nullptr, r);
}
tomo_status tomo_solve(tomo_grid* G, const float* rho, float* u, tomo_solve_info* info) {
  ENTER(G, false);
  return do_solve<float>(G, rho, u, info);
}
tomo_status tomo_solve_d(tomo_grid* G, const double* rho, double* u, tomo_solve_info* info) {
  ENTER(G, true);
  return do_solve<double>(G, rho, u, info);
}
tomo_status tomo_sensitivity(tomo_grid* G, const float* rho, const float* u, double* c,
                             float* dc) {
  ENTER(G, false);
  return do_sensitivity<float>(G, rho, u, c, dc);
}
tomo_status tomo_sensitivity_d(tomo_grid* G, const double* rho, const double* u, double* c,
                               double* dc) {
  ENTER(G, true);
  return do_sensitivity<double>(G, rho, u, c, dc);
}
tomo_status tomo_oc_step(tomo_grid* G, const float* z, const float* dcdz, const float* dvdz,
                         double volfrac, double move, float* z_new, double* change) {
  ENTER(G, false);
  return do_oc<float>(G, z, dcdz, dvdz, volfrac, move, z_new, change);
}
tomo_status tomo_oc_step_d(tomo_grid* G, const double* z, const double* dcdz, const double* dvdz,
                           double volfrac, double move, double* z_new, double* change) {
  ENTER(G, true);
  return do_oc<double>(G, z, dcdz, dvdz, volfrac, move, z_new, change);
}
tomo_status tomo_gradient(tomo_grid* G, const float* z, double* c, float* dcdz, float* dvdz,
                          tomo_solve_info* info) {
  ENTER(G, false);
  return do_gradient<float>(G, z, c, dcdz, dvdz, info);
}
tomo_status tomo_gradient_d(tomo_grid* G, const double* z, double* c, double* dcdz,
                            double* dvdz, tomo_solve_info* info) {
  ENTER(G, true);
  return do_gradient<double>(G, z, c, dcdz, dvdz, info);
}
tomo_status tomo_get_displacement(tomo_grid* G, float* u) {
  ENTER(G, false);
  return do_get_u<float>(G, u);
}
tomo_status tomo_get_displacement_d(tomo_grid* G, double* u) {
  ENTER(G, true);
  return do_get_u<double>(G, u);
}

tomo_status tomo_get_counts(const tomo_grid* G, int64_t* n_el, int64_t* n_nodes,
                            int32_t* mg_levels) {
  if (!G) return TOMO_EINVAL;
  if (n_el) *n_el = G->g.nel;
  if (n_nodes) *n_nodes = G->g.nn;
  if (mg_levels) *mg_levels = (int32_t)G->L.size();
  return TOMO_OK;
}

tomo_status tomo_get_launch_count(const tomo_grid* G, int64_t* launches) {
  if (!G || !launches) return TOMO_EINVAL;
  *launches = G->launches;
  return TOMO_OK;
}

tomo_status tomo_profile_enable(tomo_grid* G, int enable) {
  if (!G) return TOMO_EINVAL;
  G->prof = (enable & 1) != 0;
  G->phase_prof = (enable & 2) != 0;
  return TOMO_OK;
}

tomo_status tomo_profile_levels(tomo_grid* G, double* ms, int64_t* launches, int max_levels) {
  if (!G || !ms || max_levels < 1) return TOMO_EINVAL;
  for (int l = 0; l < max_levels && l < 16; ++l) {
    ms[l] = G->level_ms[l];
    if (launches) launches[l] = G->level_n[l];
    G->level_ms[l] = 0.0;
    G->level_n[l] = 0;
  }
  return TOMO_OK;
}

tomo_status tomo_profile_phases(tomo_grid* G, double* ms, int64_t* calls) {
  if (!G || !ms) return TOMO_EINVAL;
  for (int i = 0; i < 7; ++i) {
    ms[i] = G->phase_ms[i];
    G->phase_ms[i] = 0.0;
  }
  if (calls) *calls = G->phase_calls;
  G->phase_calls = 0;
  return TOMO_OK;
}

tomo_status tomo_profile_read(tomo_grid* G, int64_t* launches, double* total_ms,
                              double* algorithmic_bytes) {
  if (!G) return TOMO_EINVAL;
  G->err.clear();
  g_cur_err = &G->err;
  TRY(sync(G));
  double ms = 0.0;
  for (size_t q = 0; q + 1 < G->ev_used; q += 2) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, G->ev[q], G->ev[q + 1]));
    const int tag = (q / 2 < G->ev_tag.size()) ? G->ev_tag[q / 2] : -1;
    if (tag == -2) continue;  // enqueued after the solve stopped: no work
    if (tag < 0) {
      ms += t;
      G->prof_launches += 1;
      G->prof_bytes += G->ev_bytes[q / 2];
      G->level_ms[0] += t;
      G->level_n[0] += 1;
    } else if (tag - 1 < 16) {
      G->level_ms[tag - 1] += t;
      G->level_n[tag - 1] += 1;
    }
  }
  if (launches) *launches = G->prof_launches;
  if (total_ms) *total_ms = ms;
  if (algorithmic_bytes) *algorithmic_bytes = G->prof_bytes;
  G->ev_used = 0;
  G->prof_launches = 0;
  G->prof_bytes = 0.0;
  return TOMO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batches: many independent grids evaluated together.  Small grids leave most of the GPU
// idle, and their CG loops are bound by the launch rate (a V-cycle is ~6 short launches per
// level), so a batch runs in lockstep: per-grid setup on `workers` host threads with a
// stream each (largest grids first), then ONE CG loop for all grids in which every phase of
// an iteration (the product, the vector updates, each level's smoothing, transfer and
// coarse solve) is one launch covering every grid, captured once as a conditional-while
// graph; then per-grid sensitivities on the worker streams.  Each grid gets the tiles and
// blocks of its own single-grid launches; only the z-chunks of the products are chosen for
// the batch (one wave for all grids together), which changes the order in which the fused
// dots (p.q, r.z) add their block partials, so a grid's result agrees with its result alone
// to rounding (and is reproducible for the same batch).  Grids that cannot share a loop
// (FP64, Jacobi preconditioner, profiling, different smoother settings or Poisson ratios)
// run one per worker stream instead, bitwise as alone.
// ---------------------------------------------------------------------------------------
struct tomo_batch {
  std::vector<tomo_grid*> grids;
  std::vector<cudaStream_t> streams;
  int device = 0;  // device of the worker streams (current at creation)
  std::string err;
  bool lockstep = true;
  int64_t lockstep_runs = 0;
  // captured lockstep loop of the active grid set `plan` (with the grids' setting generations)
  std::vector<tomo_grid*> plan;
  std::vector<int64_t> plan_gen;
  cudaStream_t bst = nullptr;  // stream of the batched launches
  cudaStream_t cap = nullptr;  // capture stream
  cudaGraphExec_t loop = nullptr;
  CgScalars** d_scs = nullptr;
  int d_scs_n = 0;
  int64_t iter_launches = 0;  // batched launches per loop iteration
  std::vector<cudaEvent_t> wev;
  cudaEvent_t bev = nullptr;
  // phase timing of the last lockstep call: host ms of phase A (enqueue) and phase C
  // (results), device ms from the end of phase A to the end of the first V-cycle, of the CG
  // loop, and of the scalar read-back (events on the batch stream)
  cudaEvent_t tev[4] = {};
  double phase_ms[5] = {};
  // tiles of the batched products: thread rows per CTA (8 or 4) and the waves of resident
  // CTAs the z-chunking aims at (tomo_batch_set_tiles / tomo_batch_autotune_tiles)
  int tile_ty = 8;
  int waves = 4;
  // persistent lockstep iteration: requested, and whether the captured loop uses it
  bool persistent = false;
  bool persist_used = false;
  long long wait_limit_ns = 2000000000LL;
  int64_t persistent_runs = 0;
  unsigned char* d_tab = nullptr;  // phase tables (device)
  size_t d_tab_cap = 0;
  DevPhase* d_ph = nullptr;
  int d_ph_cap = 0;
  unsigned* d_bar = nullptr;  // grid barrier words (count, generation)
  bool persist_timing = false;             // per-phase device time accumulated
  unsigned long long* d_acc = nullptr;     // per-phase ns and launch count of the last call
  int d_acc_cap = 0;
  std::vector<int> persist_kinds;          // phase kinds of the captured iteration
  int persist_nph = 0, persist_ctas_n = 0;
  size_t persist_smem = 0;
};

namespace {

#define BK(...)                                                                      \
  do {                                                                               \
    cudaError_t _e = (__VA_ARGS__);                                                  \
    if (_e != cudaSuccess) {                                                         \
      char _b[256];                                                                  \
      std::snprintf(_b, sizeof _b, "CUDA error %d (%s) in %s", (int)_e,              \
                    cudaGetErrorString(_e), #__VA_ARGS__);                           \
      B->err = _b;                                                                   \
      return TOMO_ECUDA;                                                             \
    }                                                                                \
  } while (0)

March2Const march2_const(const tomo_grid* G) {
  return March2Const{(float)G->kinds.a0, (float)G->kinds.b0, (float)G->kinds.a7,
                     (float)G->kinds.b7, (float)G->kinds.ta, (float)G->kinds.tb,
                     (float)G->kinds.ua, (float)G->kinds.ud, (float)G->k0diag};
}

// the k_march2 arguments march() would build for this grid and level
March2Args march2_args(const tomo_grid* G, int level, const float* x, const float* b,
                       float* xprev, float* y, float c1, float c2, int dot_kind,
                       int xprev_zero) {
  const tomo_level& Lv = G->L[level];
  March2Args m{};
  m.g = Lv.g;
  m.s = (const float*)Lv.s;
  m.mask = Lv.mask;
  m.x = x;
  m.b = b;
  m.xprev = xprev;
  m.y = y;
  m.c1 = c1;
  m.c2 = c2;
  m.partials = G->partials;
  m.counter = G->counter;
  m.sc = G->sc;
  m.dot_kind = dot_kind;
  m.skip = &G->sc->done;
  m.xprev_zero = xprev_zero;
  m.tile_fixed = Lv.tile_fixed;
  m.invd = (const float*)Lv.invd;
  return m;
}

// Can these grids share one lockstep loop?  (Same launch sequence and shared constants.)
bool lockstep_compatible(const std::vector<tomo_grid*>& Gs) {
  if (Gs.empty()) return false;
  const tomo_grid* A = Gs[0];
  for (const tomo_grid* G : Gs) {
    if (G->prec != TOMO_FP32 || G->d.precond != TOMO_PRECOND_MG || !G->use_graph || G->prof ||
        G->phase_prof || G->rhs_id != 0 || G->L.size() < 2 || !G->fuse_j0 || G->wlevels != 0)
      return false;  // (the lockstep V-cycle has no W-cycle levels)
    if (G->d.smoother_degree != A->d.smoother_degree ||
        G->d.coarse_degree != A->d.coarse_degree || G->d.rr_every != A->d.rr_every ||
        G->k0diag != A->k0diag || std::memcmp(G->blk, A->blk, sizeof G->blk) != 0 ||
        std::memcmp(&G->kinds, &A->kinds, sizeof G->kinds) != 0)
      return false;
    if (G->d.rr_every > 0 && !G->s64) return false;
  }
  return true;
}

// z-chunk length (node planes per CTA) for the grids P of a batched product on `level`:
// the shortest chunks whose CTAs across the batch fit in `waves` waves of resident CTAs
// (2 per SM at 8 thread rows, 4 at 4).  A grid alone chunks for the GPU it fills by itself;
// in a batch the grids together fill it.  One wave of whole columns leaves the tallest
// grid's column as the makespan, very short chunks add halo layers and waves; measured on
// 64 uneven cantilevers at 8 rows, the CG loop took 6.79 / 6.88 / 6.63 ms with one / two /
// four waves (the default; tomo_batch_autotune_tiles measures the choice per batch).
int lockstep_kz(const std::vector<tomo_grid*>& Gs, const std::vector<int>& P, int level,
                int ty, int waves) {
  const int per_sm = ty == 4 ? 4 : 2;
  const int target = waves * per_sm * (Gs[0]->num_sms > 0 ? Gs[0]->num_sms : 152);
  int kmax = 1;
  for (int q : P) kmax = std::max(kmax, Gs[q]->L[level].g.nzn);
  for (int kz = 1; kz < kmax; ++kz) {
    long long ctas = 0;
    for (int q : P) {
      const Geom& g = Gs[q]->L[level].g;
      const long long tiles =
          (long long)((g.nxn + 29) / 30) * ((g.nyn + 2 * ty - 3) / (2 * ty - 2));
      ctas += tiles * ((g.nzn + kz - 1) / kz);
    }
    if (ctas <= target) return kz;
  }
  return kmax;
}

struct ChebCoef {
  float c1, c2;
};

// Chebyshev coefficients of steps 0..K-1 of one grid (as smooth() computes them)
std::vector<ChebCoef> cheb_steps(const tomo_grid* G, int K) {
  const Cheb cb = cheb(G);
  std::vector<ChebCoef> v(K);
  double rho_prev = 1.0 / cb.sigma;
  for (int s = 0; s < K; ++s) {
    double c1, c2;
    if (s == 0) {
      c1 = 0.0;
      c2 = 1.0 / cb.theta;
    } else {
      const double rho = 1.0 / (2.0 * cb.sigma - rho_prev);
      c1 = rho * rho_prev;
      c2 = 2.0 * rho / cb.delta;
      rho_prev = rho;
    }
    v[s] = ChebCoef{(float)c1, (float)c2};
  }
  return v;
}

// z = V-cycle(r) for every grid of Gs, the same sequence vcycle() issues per grid, with each
// operation issued once for all grids that have it (a grid's coarsest solve after the
// batch's down-sweep: nothing of that grid runs in between).  dot: the last smoothing step
// on level 0 computes r.z (beta).  *launches counts the batched launches issued.
tomo_status batch_vcycle(tomo_batch* B, cudaStream_t st, const std::vector<tomo_grid*>& Gs,
                         const std::vector<const float*>& rin, bool dot,
                         std::vector<float*>* zout, int64_t* launches,
                         bool first_done0 = false) {
  const int n = (int)Gs.size();
  const tomo_grid* G0 = Gs[0];
  const March2Const kc = march2_const(G0);
  const int num_sms = G0->num_sms;
  int Lmax = 0;
  for (auto* G : Gs) Lmax = std::max(Lmax, (int)G->L.size());
  std::vector<std::vector<float*>> X(n), Y(n);
  for (int q = 0; q < n; ++q) {
    const int nl = (int)Gs[q]->L.size();
    X[q].resize(nl);
    Y[q].resize(nl);
    for (int l = 0; l < nl; ++l) {
      X[q][l] = (float*)Gs[q]->L[l].x;
      Y[q][l] = (float*)Gs[q]->L[l].xp;
    }
  }
  auto rhs = [&](int q, int l) -> const float* {
    return l == 0 ? rin[q] : (const float*)Gs[q]->L[l].b;
  };
  std::vector<int> P;
  std::vector<March2Args> ma;
  auto part = [&](int l) {  // grids for which level l is not the coarsest
    P.clear();
    for (int q = 0; q < n; ++q)
      if (l < (int)Gs[q]->L.size() - 1) P.push_back(q);
  };
  auto cheb_step = [&](int l, int s, const std::vector<std::vector<ChebCoef>>& cf,
                       bool zero_start, int dk) -> tomo_status {
    ma.clear();
    const int kz = lockstep_kz(Gs, P, l, B->tile_ty, B->waves);
    for (int q : P) {
      ma.push_back(march2_args(Gs[q], l, X[q][l], rhs(q, l), Y[q][l], nullptr, cf[q][s].c1,
                               cf[q][s].c2, dk, (s == 1 && zero_start) ? 1 : 0));
      ma.back().kz = kz;
    }
    BK(launch_march2_batch(st, M_CHEB, ma.data(), (int)ma.size(), kc, num_sms, B->tile_ty));
    *launches += 1;
    for (int q : P) std::swap(X[q][l], Y[q][l]);
    return TOMO_OK;
  };
  // down-sweep
  for (int l = 0; l + 1 < Lmax; ++l) {
    part(l);
    if (P.empty()) continue;
    const int K = level_degree(G0, l);
    std::vector<std::vector<ChebCoef>> cf(n);
    for (int q : P) cf[q] = cheb_steps(Gs[q], K);
    for (int s = 0; s < K; ++s) {
      if (s == 0) {
        // (levels >= 1: the restriction that produced b wrote x1; level 0 inside the loop:
        // the CG update did)
        if (l == 0 && !first_done0) {
          std::vector<JacobiItem> ja;
          for (int q : P) {
            const tomo_level& Lv = Gs[q]->L[0];
            ja.push_back(JacobiItem{Lv.g, (const float*)Lv.s, Lv.mask, rhs(q, 0), cf[q][0].c2,
                                    (float)Gs[q]->k0diag, X[q][0], &Gs[q]->sc->done,
                                    nullptr});
          }
          BK(launch_jacobi_batch(st, ja.data(), (int)ja.size()));
          *launches += 1;
        }
        continue;
      }
      TRY(cheb_step(l, s, cf, true, 0));
    }
    ma.clear();
    const int kz = lockstep_kz(Gs, P, l, B->tile_ty, B->waves);
    for (int q : P) {
      ma.push_back(march2_args(Gs[q], l, X[q][l], rhs(q, l), nullptr,
                               (float*)Gs[q]->L[l].t, 0.0f, 0.0f, 0, 0));
      ma.back().kz = kz;
    }
    BK(launch_march2_batch(st, M_RESID, ma.data(), (int)ma.size(), kc, num_sms, B->tile_ty));
    *launches += 1;
    std::vector<RestrictItem> ra;
    for (int q : P) {
      const tomo_grid* G = Gs[q];
      const tomo_level& Lv = G->L[l];
      const tomo_level& Lc = G->L[l + 1];
      const bool fuse = l + 1 < (int)G->L.size() - 1;
      ra.push_back(RestrictItem{Lv.g, Lc.g, (const float*)Lv.t, (float*)Lc.b, Lc.mask,
                                &G->sc->done, fuse ? (float*)Lc.x : nullptr,
                                (const float*)Lc.s, (float)(1.0 / cheb(G).theta),
                                (float)G->k0diag});
    }
    BK(launch_restrict_batch(st, ra.data(), (int)ra.size()));
    *launches += 1;
  }
  // coarsest levels
  std::vector<float*> zc(n);
  {
    std::vector<CoarseItem> ca;
    for (int q = 0; q < n; ++q) {
      const tomo_grid* G = Gs[q];
      const int lc = (int)G->L.size() - 1;
      zc[q] = (float*)G->L[lc].x;
      ca.push_back(CoarseItem{G->coarse_n, (const float*)G->coarseA, (const float*)G->coarseD,
                              rhs(q, lc), zc[q], &G->sc->done});
    }
    BK(launch_coarse_apply_batch(st, ca.data(), n));
    *launches += 1;
  }
  // up-sweep
  for (int l = Lmax - 2; l >= 0; --l) {
    part(l);
    if (P.empty()) continue;
    std::vector<ProlongItem> pa;
    for (int q : P) {
      const tomo_level& Lv = Gs[q]->L[l];
      pa.push_back(ProlongItem{Lv.g, Gs[q]->L[l + 1].g, zc[q], X[q][l], Lv.mask,
                               &Gs[q]->sc->done});
    }
    BK(launch_prolong_batch(st, pa.data(), (int)pa.size()));
    *launches += 1;
    const int K = level_degree(G0, l);
    std::vector<std::vector<ChebCoef>> cf(n);
    for (int q : P) cf[q] = cheb_steps(Gs[q], K);
    for (int s = 0; s < K; ++s)
      TRY(cheb_step(l, s, cf, false, (dot && l == 0 && s == K - 1) ? 2 : 0));
    for (int q : P) zc[q] = X[q][l];
  }
  *zout = zc;
  return TOMO_OK;
}

tomo_status batch_cg_p(tomo_batch* B, cudaStream_t st, const std::vector<tomo_grid*>& Gs,
                       const std::vector<float*>& z, int64_t* launches) {
  std::vector<CgPItem> pa;
  for (size_t q = 0; q < Gs.size(); ++q)
    pa.push_back(CgPItem{3 * Gs[q]->g.nn, (float*)Gs[q]->p, z[q], Gs[q]->sc});
  BK(launch_cg_p_batch(st, pa.data(), (int)pa.size()));
  *launches += 1;
  return TOMO_OK;
}

// One CG iteration for every grid (enqueue_iteration's sequence, batched).
tomo_status batch_iteration(tomo_batch* B, cudaStream_t st, const std::vector<tomo_grid*>& Gs,
                            int64_t* launches) {
  const int n = (int)Gs.size();
  const tomo_grid* G0 = Gs[0];
  std::vector<March2Args> ma;
  std::vector<int> all(n);
  for (int q = 0; q < n; ++q) all[q] = q;
  const int kz = lockstep_kz(Gs, all, 0, B->tile_ty, B->waves);
  for (auto* G : Gs) {
    ma.push_back(march2_args(G, 0, (const float*)G->p, nullptr, nullptr, (float*)G->q, 0.0f,
                             0.0f, 1, 0));
    ma.back().kz = kz;
  }
  BK(launch_march2_batch(st, M_APPLY, ma.data(), n, march2_const(G0), G0->num_sms,
                         B->tile_ty));
  *launches += 1;
  // every lockstep grid is an FP32 multigrid grid, so all have the fused first step
  std::vector<CgXrItem> xa;
  for (auto* G : Gs)
    xa.push_back(CgXrItem{3 * G->g.nn, (float*)G->xhi, (float*)G->xlo, (float*)G->r,
                          (const float*)G->p, (const float*)G->q, G->partials, G->counter,
                          G->sc, (float*)G->L[0].x, (const float*)G->invd,
                          (float)(1.0 / cheb(G).theta)});
  BK(launch_cg_xr_batch(st, xa.data(), n));
  *launches += 1;
  if (G0->d.rr_every > 0) {
    std::vector<MarchArgs<double>> ra;
    for (auto* G : Gs) {
      MarchArgs<double> rr{};
      rr.g = G->L[0].g;
      rr.s = G->s64;
      rr.mask = G->L[0].mask;
      rr.partials = G->partials;
      rr.counter = G->counter;
      rr.xf_hi = (const float*)G->xhi;
      rr.xf_lo = (const float*)G->xlo;
      rr.b = G->rhs64;
      rr.yf = (float*)G->r;
      rr.skip = &G->sc->done;
      rr.gate = G->sc;
      rr.x1f = (float*)G->L[0].x;
      rr.invdf = (const float*)G->invd;
      rr.c2f = (float)(1.0 / cheb(G).theta);
      ra.push_back(rr);
    }
    BK(launch_march_rr_batch(st, ra.data(), n, elem_const<double>(G0), G0->num_sms));
    *launches += 1;
  }
  std::vector<const float*> r(n);
  for (int q = 0; q < n; ++q) r[q] = (const float*)Gs[q]->r;
  std::vector<float*> z;
  TRY(batch_vcycle(B, st, Gs, r, true, &z, launches, true));
  return batch_cg_p(B, st, Gs, z, launches);
}

// Record one lockstep iteration's batched launches as the phases of the persistent kernel
// (nothing is launched while recording) and upload the phase list and tables, ordered on
// the batch stream before the loop's next launch.  *ok = false: the device cannot hold the
// kernel's CTAs co-resident (the caller keeps the launched iteration).
tomo_status batch_record_persist(tomo_batch* B, const std::vector<tomo_grid*>& Gs, bool* ok) {
  *ok = false;
  if (B->tile_ty != 8) return TOMO_OK;  // the persistent units are 8-row product tiles
  std::vector<PhaseRec> rec;
  int64_t unused = 0;
  g_phase_rec = &rec;
  const tomo_status s = batch_iteration(B, B->bst, Gs, &unused);
  g_phase_rec = nullptr;
  if (s != TOMO_OK) return s;
  std::vector<DevPhase> ph;
  std::vector<std::vector<UnitDesc>> units(rec.size());
  size_t off = 0, smem = 0;
  for (size_t k = 0; k < rec.size(); ++k) {
    const PhaseRec& r = rec[k];
    // every table starts with the grid count and the block offsets cta0; the product
    // tables follow them with the tile counts gx, gy
    int n = 0;
    std::vector<int> cta0(kBatchMax + 1, 0);
    std::vector<short> gx(kBatchMax, 0), gy(kBatchMax, 0);
    std::memcpy(&n, r.table.data(), sizeof(int));
    std::memcpy(cta0.data(), r.table.data() + sizeof(int), sizeof(int) * (kBatchMax + 1));
    const bool prod = r.kind <= PH_RR;
    if (prod) {
      static_assert(offsetof(March2Batch, gx) == offsetof(MarchRrBatch, gx) &&
                        offsetof(March2Batch, gy) == offsetof(MarchRrBatch, gy),
                    "product tables share their head");
      std::memcpy(gx.data(), r.table.data() + offsetof(March2Batch, gx),
                  sizeof(short) * kBatchMax);
      std::memcpy(gy.data(), r.table.data() + offsetof(March2Batch, gy),
                  sizeof(short) * kBatchMax);
    }
    for (int q = 0; q < n; ++q)
      for (int b = cta0[q]; b < cta0[q + 1]; ++b)
        units[k].push_back(UnitDesc{q, b - cta0[q], cta0[q + 1] - cta0[q], gx[q], gy[q]});
    if ((int)units[k].size() != r.units) return TOMO_OK;  // not a table of this layout
    int nunits = r.units;
    if (r.kind == PH_COARSE) {
      // a grid's 1024-thread coarsest solve as four 256-thread units, each a quarter of
      // the block's warps (the persistent kernel's CTAs have 256 threads)
      std::vector<UnitDesc> four;
      for (const UnitDesc& d : units[k])
        for (int part = 0; part < 4; ++part) four.push_back(UnitDesc{d.q, part, 4, 0, 0});
      units[k].swap(four);
      nunits = (int)units[k].size();
    }
    off = (off + 255) & ~(size_t)255;
    const size_t uoff = off;
    off += sizeof(UnitDesc) * units[k].size();
    off = (off + 255) & ~(size_t)255;
    ph.push_back(DevPhase{r.kind, nunits, r.join, 0, (long long)uoff, (long long)off});
    off += r.table.size();
    if (r.kind == PH_COARSE) {
      FlatBatch<CoarseItem> t;
      std::memcpy(&t, r.table.data(), sizeof t);
      for (int q = 0; q < t.n; ++q) smem = std::max(smem, sizeof(float) * (size_t)t.a[q].n);
    }
  }
  if (ph.empty()) return TOMO_OK;
  const int ctas = persist_ctas(Gs[0]->num_sms, smem);
  if (ctas <= 0) return TOMO_OK;
  std::vector<unsigned char> host(off);
  for (size_t k = 0; k < rec.size(); ++k) {
    std::memcpy(host.data() + ph[k].units_offset, units[k].data(),
                sizeof(UnitDesc) * units[k].size());
    std::memcpy(host.data() + ph[k].offset, rec[k].table.data(), rec[k].table.size());
  }
  if (off > B->d_tab_cap) {
    if (B->d_tab) cudaFree(B->d_tab);
    B->d_tab = nullptr;
    B->d_tab_cap = 0;
    BK(cudaMalloc(&B->d_tab, off));
    B->d_tab_cap = off;
  }
  if ((int)ph.size() > B->d_ph_cap) {
    if (B->d_ph) cudaFree(B->d_ph);
    B->d_ph = nullptr;
    B->d_ph_cap = 0;
    BK(cudaMalloc(&B->d_ph, sizeof(DevPhase) * ph.size()));
    B->d_ph_cap = (int)ph.size();
  }
  if (!B->d_bar) BK(cudaMalloc(&B->d_bar, 4 * sizeof(unsigned)));
  if ((int)ph.size() + 1 > B->d_acc_cap) {
    if (B->d_acc) cudaFree(B->d_acc);
    B->d_acc = nullptr;
    B->d_acc_cap = 0;
    BK(cudaMalloc(&B->d_acc, sizeof(unsigned long long) * (ph.size() + 1)));
    B->d_acc_cap = (int)ph.size() + 1;
  }
  BK(cudaMemsetAsync(B->d_acc, 0, sizeof(unsigned long long) * (ph.size() + 1), B->bst));
  B->persist_kinds.clear();
  for (const DevPhase& d : ph) B->persist_kinds.push_back(d.kind);
  // pageable sources: each call returns once its bytes are staged
  BK(cudaMemcpyAsync(B->d_tab, host.data(), off, cudaMemcpyHostToDevice, B->bst));
  BK(cudaMemcpyAsync(B->d_ph, ph.data(), sizeof(DevPhase) * ph.size(), cudaMemcpyHostToDevice,
                     B->bst));
  B->persist_nph = (int)ph.size();
  B->persist_ctas_n = ctas;
  B->persist_smem = smem;
  *ok = true;
  return TOMO_OK;
}

// Capture the device-side CG loop (a conditional while node) whose body is one lockstep
// iteration: the persistent kernel (persist) or the batched launches, then the loop test.
tomo_status batch_capture_loop(tomo_batch* B, const std::vector<tomo_grid*>& Gs, bool persist,
                               int64_t* launches, cudaGraphExec_t* out) {
  const int n = (int)Gs.size();
  cudaGraph_t graph;
  BK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle hc;
  cudaError_t e = cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    BK(e);
  }
  e = cudaStreamBeginCaptureToGraph(B->cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  tomo_status st = TOMO_OK;
  *launches = 0;
  if (e == cudaSuccess) {
    if (persist) {
      const tomo_grid* G0 = Gs[0];
      cudaError_t e1 = launch_persist(B->cap, B->d_ph, B->persist_nph, B->d_tab,
                                      march2_const(G0), elem_const<double>(G0), B->d_bar,
                                      B->wait_limit_ns, B->d_scs, n, B->persist_ctas_n,
                                      B->persist_smem,
                                      B->persist_timing ? B->d_acc : nullptr);
      *launches += 1;
      if (e1 != cudaSuccess) {
        B->err = std::string("persistent iteration launch failed: ") + cudaGetErrorString(e1);
        st = TOMO_ECUDA;
      }
    } else {
      st = batch_iteration(B, B->cap, Gs, launches);
    }
    if (st == TOMO_OK) {
      cudaError_t e2 = launch_loop_cond_batch(B->cap, hc, B->d_scs, n);
      *launches += 1;
      if (e2 != cudaSuccess) {
        B->err = std::string("loop control launch failed: ") + cudaGetErrorString(e2);
        st = TOMO_ECUDA;
      }
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(B->cap, &captured);
    if (st == TOMO_OK && e3 != cudaSuccess) e = e3;
  }
  if (e != cudaSuccess || st != TOMO_OK) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != TOMO_OK) return st;
    BK(e);
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  BK(e);
  return TOMO_OK;
}

tomo_status batch_build_loop(tomo_batch* B, const std::vector<tomo_grid*>& Gs) {
  if (B->loop) {
    cudaGraphExecDestroy(B->loop);
    B->loop = nullptr;
  }
  B->persist_used = false;
  const int n = (int)Gs.size();
  if (B->d_scs_n < n) {
    if (B->d_scs) cudaFree(B->d_scs);
    B->d_scs = nullptr;
    B->d_scs_n = 0;
    BK(cudaMalloc(&B->d_scs, sizeof(CgScalars*) * (size_t)n));
    B->d_scs_n = n;
  }
  std::vector<CgScalars*> h(n);
  for (int q = 0; q < n; ++q) h[q] = Gs[q]->sc;
  BK(cudaMemcpyAsync(B->d_scs, h.data(), sizeof(CgScalars*) * (size_t)n, cudaMemcpyHostToDevice,
                     B->bst));
  if (!B->cap) BK(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  int64_t launches = 0;
  if (B->persistent) {
    bool ok = false;
    TRY(batch_record_persist(B, Gs, &ok));
    if (ok) {
      const tomo_status s = batch_capture_loop(B, Gs, true, &launches, &B->loop);
      if (s == TOMO_OK) {
        B->persist_used = true;
      } else if (s == TOMO_ECUDA) {  // not capturable here: the launched iteration
        cudaGetLastError();
        B->err.clear();
      } else {
        return s;
      }
    }
  }
  if (!B->persist_used) TRY(batch_capture_loop(B, Gs, false, &launches, &B->loop));
  B->plan = Gs;
  B->plan_gen.clear();
  for (auto* G : Gs) B->plan_gen.push_back(G->gen);
  B->iter_launches = launches;
  return TOMO_OK;
}

// Run fn(w, i) for every grid index i on W worker threads, largest grids first, each grid
// taken by the next free worker.
template <class Fn>
void for_grids_lpt(tomo_batch* B, int W, Fn fn) {
  const int n = (int)B->grids.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return B->grids[a]->g.nel > B->grids[b]->g.nel;
  });
  std::atomic<int> next{0};
  auto work = [&](int w) {
    // a new host thread starts on device 0: select the batch's device first
    if (w > 0 && cudaSetDevice(B->device) != cudaSuccess) cudaGetLastError();
    for (int k = next++; k < n; k = next++) fn(w, order[k]);
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < W; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
}

tomo_status batch_first_error(tomo_batch* B, const std::vector<tomo_status>& st) {
  for (size_t i = 0; i < st.size(); ++i)
    if (st[i] != TOMO_OK) {
      char buf[64];
      std::snprintf(buf, sizeof buf, "grid %d of the batch: ", (int)i);
      B->err = std::string(buf) + B->grids[i]->err;
      return st[i];
    }
  return TOMO_OK;
}

tomo_status batch_lockstep(tomo_batch* B, const float* const* z, double* compliance,
                           float* const* dcdz, float* const* dvdz, tomo_solve_info* info) {
  const int n = (int)B->grids.size();
  const int W = std::min<int>((int)B->streams.size(), std::max(n, 1));
  if (!B->bst) BK(cudaStreamCreateWithFlags(&B->bst, cudaStreamNonBlocking));
  while ((int)B->wev.size() < W) {
    cudaEvent_t e;
    BK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B->wev.push_back(e);
  }
  if (!B->bev) BK(cudaEventCreateWithFlags(&B->bev, cudaEventDisableTiming));
  std::vector<tomo_status> st(n, TOMO_OK);
  std::vector<GradIO> io(n);
  std::vector<char> trivial(n, 0);
  std::vector<cudaStream_t> own(n);
  for (int i = 0; i < n; ++i) own[i] = B->grids[i]->stream;
  for (auto& e : B->tev)
    if (!e) BK(cudaEventCreate(&e));
  const auto h0 = std::chrono::steady_clock::now();
  // phase A: S1-S2 and the CG start of every grid, on the worker streams
  for_grids_lpt(B, W, [&](int w, int i) {
    tomo_grid* G = B->grids[i];
    G->stream = B->streams[w];
    g_cur_err = &G->err;
    G->err.clear();
    st[i] = gradient_begin<float>(G, z[i], dcdz[i], dvdz ? dvdz[i] : nullptr, &io[i]);
    bool tv = false;
    if (st[i] == TOMO_OK)
      st[i] = pcg_start<float>(G, G->warm_gradient && G->have_solution,
                               info ? info + i : nullptr, &tv);
    trivial[i] = tv ? 1 : 0;
  });
  for (int w = 0; w < W; ++w) {
    BK(cudaEventRecord(B->wev[w], B->streams[w]));
    BK(cudaStreamWaitEvent(B->bst, B->wev[w], 0));
  }
  // the coarsest factorisations run concurrently on the grids' side streams; the batch
  // stream (first coarsest solve) waits for each of them, not the worker streams
  for (int i = 0; i < n; ++i) {
    tomo_grid* G = B->grids[i];
    if (G->factor_pending) {
      G->factor_pending = false;
      BK(cudaStreamWaitEvent(B->bst, G->ev_factor, 0));
    }
  }
  const auto h1 = std::chrono::steady_clock::now();
  BK(cudaEventRecord(B->tev[0], B->bst));
  // phase B: one CG loop for the grids that have a system to solve
  NvtxRange range_b("tomo batch: lockstep CG loop");
  std::vector<tomo_grid*> act;
  for (int i = 0; i < n; ++i)
    if (st[i] == TOMO_OK && !trivial[i]) act.push_back(B->grids[i]);
  tomo_status bs = TOMO_OK;
  if (!act.empty()) {
    int64_t launches = 0;
    std::vector<const float*> r(act.size());
    for (size_t q = 0; q < act.size(); ++q) r[q] = (const float*)act[q]->r;
    std::vector<float*> zz;
    bs = batch_vcycle(B, B->bst, act, r, true, &zz, &launches);
    if (bs == TOMO_OK) bs = batch_cg_p(B, B->bst, act, zz, &launches);
    if (bs == TOMO_OK && cudaEventRecord(B->tev[1], B->bst) != cudaSuccess) bs = TOMO_ECUDA;
    bool stale = !B->loop || B->plan != act;
    for (size_t q = 0; !stale && q < act.size(); ++q) stale = B->plan_gen[q] != act[q]->gen;
    if (bs == TOMO_OK && stale) bs = batch_build_loop(B, act);
    if (bs == TOMO_OK) {
      cudaError_t e = cudaSuccess;
      if (B->persist_used)  // barrier words from zero (a timed-out call leaves them mid-count)
        e = cudaMemsetAsync(B->d_bar, 0, 4 * sizeof(unsigned), B->bst);
      if (e == cudaSuccess && B->persist_used && B->persist_timing)
        e = cudaMemsetAsync(B->d_acc, 0, sizeof(unsigned long long) * (B->persist_nph + 1),
                            B->bst);
      const bool injected = e == cudaSuccess && fault_hit(FAULT_GRAPH);
      if (e == cudaSuccess && !injected) e = cudaGraphLaunch(B->loop, B->bst);
      if (e == cudaSuccess) e = cudaEventRecord(B->tev[2], B->bst);
      for (size_t q = 0; q < act.size() && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(act[q]->h_sc, act[q]->sc, sizeof(CgScalars),
                            cudaMemcpyDeviceToHost, B->bst);
      if (e == cudaSuccess) e = cudaEventRecord(B->tev[3], B->bst);
      if (e == cudaSuccess) e = cudaStreamSynchronize(B->bst);
      if (e != cudaSuccess) {
        B->err = std::string("lockstep CG loop: ") + cudaGetErrorString(e);
        bs = TOMO_ECUDA;
      } else if (injected) {
        B->err = "injected CG loop launch failure";
        bs = TOMO_ECUDA;
      }
      float t01 = 0.f, t12 = 0.f, t23 = 0.f;
      if (bs == TOMO_OK) {
        cudaEventElapsedTime(&t01, B->tev[0], B->tev[1]);
        cudaEventElapsedTime(&t12, B->tev[1], B->tev[2]);
        cudaEventElapsedTime(&t23, B->tev[2], B->tev[3]);
        cudaGetLastError();
      }
      B->phase_ms[1] = t01;
      B->phase_ms[2] = t12;
      B->phase_ms[3] = t23;
    }
    if (bs == TOMO_OK) {
      for (auto* G : act) G->launches += launches + (int64_t)G->h_sc->loops * B->iter_launches;
      if (B->persist_used) B->persistent_runs += 1;
    }
  }
  const auto h2 = std::chrono::steady_clock::now();
  if (bs == TOMO_OK) {
    BK(cudaEventRecord(B->bev, B->bst));
    // phase C: results, S6-S7 on the worker streams
    for_grids_lpt(B, W, [&](int w, int i) {
      if (st[i] != TOMO_OK) return;
      tomo_grid* G = B->grids[i];
      G->stream = B->streams[w];
      g_cur_err = &G->err;
      // after every grid's phase A (the batch stream waited for all of it) and the loop
      if (cudaStreamWaitEvent(G->stream, B->bev, 0) != cudaSuccess) {
        cudaGetLastError();
        st[i] = fail(G, TOMO_ECUDA, "stream wait failed");
        return;
      }
      if (!trivial[i]) st[i] = pcg_result(G, info ? info + i : nullptr);
      if (st[i] == TOMO_OK)
        st[i] = gradient_end<float>(G, io[i], compliance + i, dcdz[i],
                                    dvdz ? dvdz[i] : nullptr, true);
    });
    // one synchronisation per worker stream, then the compliances
    for (int w = 0; w < W; ++w)
      if (cudaStreamSynchronize(B->streams[w]) != cudaSuccess) {
        cudaGetLastError();
        for (int i = 0; i < n; ++i)
          if (st[i] == TOMO_OK) st[i] = fail(B->grids[i], TOMO_ECUDA, "batch stream failed");
        break;
      }
    for (int i = 0; i < n; ++i)
      if (st[i] == TOMO_OK && !is_device_ptr(compliance + i)) compliance[i] = *B->grids[i]->h_scal;
  }
  const auto h3 = std::chrono::steady_clock::now();
  B->phase_ms[0] = std::chrono::duration<double, std::milli>(h1 - h0).count();
  B->phase_ms[4] = std::chrono::duration<double, std::milli>(h3 - h2).count();
  // the worker streams must not run ahead of anything still queued on the batch stream
  cudaStreamSynchronize(B->bst);
  for (int i = 0; i < n; ++i) B->grids[i]->stream = own[i];
  if (bs != TOMO_OK) return bs;
  B->lockstep_runs += 1;
  return batch_first_error(B, st);
}

}  // namespace

extern "C" {

tomo_status tomo_batch_create(int32_t workers, tomo_batch** out) {
  if (!out) return TOMO_EINVAL;
  *out = nullptr;
  if (workers <= 0) workers = 8;
  if (workers > 64) workers = 64;
  tomo_batch* B = new (std::nothrow) tomo_batch();
  if (!B) return TOMO_ENOMEM;
  if (cudaGetDevice(&B->device) != cudaSuccess) {
    cudaGetLastError();
    delete B;
    g_create_err = "tomo_batch_create: no usable CUDA device";
    return TOMO_ECUDA;
  }
  for (int w = 0; w < workers; ++w) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto t : B->streams) cudaStreamDestroy(t);
      delete B;
      g_create_err = "tomo_batch_create: stream creation failed";
      return TOMO_ECUDA;
    }
    B->streams.push_back(s);
  }
  *out = B;
  return TOMO_OK;
}

tomo_status tomo_batch_append(tomo_batch* B, tomo_grid* G) {
  if (!B || !G) return TOMO_EINVAL;
  if (G->device != B->device) {
    B->err = "the grid lives on another device than the batch's streams";
    return TOMO_EINVAL;
  }
  for (auto* q : B->grids)
    if (q == G) {
      B->err = "grid appended twice";
      return TOMO_EINVAL;
    }
  B->grids.push_back(G);
  B->plan.clear();  // the captured lockstep loop no longer covers the batch
  return TOMO_OK;
}

tomo_status tomo_batch_set_lockstep(tomo_batch* B, int32_t on) {
  if (!B) return TOMO_EINVAL;
  B->lockstep = on != 0;
  return TOMO_OK;
}

tomo_status tomo_batch_set_persistent(tomo_batch* B, int32_t on) {
  if (!B || on < 0 || on > 2) return TOMO_EINVAL;
  if (B->persistent != (on != 0) || B->persist_timing != (on == 2))
    B->plan.clear();  // recapture the loop
  B->persistent = on != 0;
  B->persist_timing = on == 2;
  return TOMO_OK;
}

tomo_status tomo_batch_set_wait_limit(tomo_batch* B, int64_t limit_ns) {
  if (!B || limit_ns < 0) return TOMO_EINVAL;
  if (B->wait_limit_ns != limit_ns) B->plan.clear();  // the limit is a launch argument
  B->wait_limit_ns = limit_ns;
  return TOMO_OK;
}

tomo_status tomo_batch_persistent_info(const tomo_batch* B, int32_t* ctas, int32_t* phases,
                                       int64_t* runs) {
  if (!B) return TOMO_EINVAL;
  if (ctas) *ctas = B->persist_used ? B->persist_ctas_n : 0;
  if (phases) *phases = B->persist_used ? B->persist_nph : 0;
  if (runs) *runs = B->persistent_runs;
  return TOMO_OK;
}

tomo_status tomo_batch_persistent_phase_ns(tomo_batch* B, int64_t* ns, int32_t* kinds,
                                           int32_t cap, int32_t* count, int64_t* launches) {
  if (!B || !count || cap < 0 || (cap > 0 && (!ns || !kinds))) return TOMO_EINVAL;
  const int nph = (B->persist_used && B->persist_timing) ? B->persist_nph : 0;
  *count = nph;
  if (launches) *launches = 0;
  if (nph == 0) return TOMO_OK;
  std::vector<unsigned long long> t(nph + 1);
  BK(cudaMemcpy(t.data(), B->d_acc, sizeof(unsigned long long) * (nph + 1),
                cudaMemcpyDeviceToHost));
  if (launches) *launches = (int64_t)t[nph];
  for (int p = 0; p < std::min(nph, (int)cap); ++p) {
    ns[p] = (int64_t)t[p];
    kinds[p] = B->persist_kinds[p];
  }
  return TOMO_OK;
}

tomo_status tomo_batch_phase_times(const tomo_batch* B, double* ms) {
  if (!B || !ms) return TOMO_EINVAL;
  for (int k = 0; k < 5; ++k) ms[k] = B->phase_ms[k];
  return TOMO_OK;
}

tomo_status tomo_batch_lockstep_runs(const tomo_batch* B, int64_t* runs) {
  if (!B || !runs) return TOMO_EINVAL;
  *runs = B->lockstep_runs;
  return TOMO_OK;
}

tomo_status tomo_batch_gradient(tomo_batch* B, const float* const* z, double* compliance,
                                float* const* dcdz, float* const* dvdz, tomo_solve_info* info) {
  if (!B || !z || !compliance || !dcdz) return TOMO_EINVAL;
  B->err.clear();
  const int n = (int)B->grids.size();
  for (int i = 0; i < n; ++i)
    if (B->grids[i]->prec != TOMO_FP32) {
      B->err = "batch gradients take FP32 grids";
      return TOMO_EINVAL;
    }
  if (B->lockstep && lockstep_compatible(B->grids))
    return batch_lockstep(B, z, compliance, dcdz, dvdz, info);
  const int W = std::min<int>((int)B->streams.size(), std::max(n, 1));
  std::vector<tomo_status> st(n, TOMO_OK);
  // one grid per worker stream at a time, largest grids first, each taken by the next free
  // worker (longest-processing-time order balances uneven sizes); a grid's work stays on
  // one stream, so its result does not depend on which worker ran it
  for_grids_lpt(B, W, [&](int w, int i) {
    {
      tomo_grid* G = B->grids[i];
      cudaStream_t own = G->stream;
      G->stream = B->streams[w];
      g_cur_err = &G->err;
      G->err.clear();
      st[i] = do_gradient<float>(G, z[i], compliance + i, dcdz[i], dvdz ? dvdz[i] : nullptr,
                                 info ? info + i : nullptr);
      if (st[i] == TOMO_OK && cudaStreamSynchronize(G->stream) != cudaSuccess) {
        cudaGetLastError();
        st[i] = TOMO_ECUDA;
      }
      G->stream = own;
    }
  });
  return batch_first_error(B, st);
}

tomo_status tomo_batch_set_tiles(tomo_batch* B, int32_t tile_rows, int32_t waves) {
  if (!B || (tile_rows != 8 && tile_rows != 4) || waves < 1 || waves > 16) return TOMO_EINVAL;
  if (tile_rows != B->tile_ty || waves != B->waves) B->plan.clear();  // recapture the loop
  B->tile_ty = tile_rows;
  B->waves = waves;
  return TOMO_OK;
}

tomo_status tomo_batch_get_tiles(const tomo_batch* B, int32_t* tile_rows, int32_t* waves) {
  if (!B) return TOMO_EINVAL;
  if (tile_rows) *tile_rows = B->tile_ty;
  if (waves) *waves = B->waves;
  return TOMO_OK;
}

tomo_status tomo_batch_autotune_tiles(tomo_batch* B, const float* const* z, float* const* dcdz,
                                      int32_t reps, tomo_batch_tune_result* res,
                                      int32_t* best) {
  if (!B || !z || !dcdz || reps < 1 || reps > 16) return TOMO_EINVAL;
  B->err.clear();
  const int n = (int)B->grids.size();
  for (int i = 0; i < n; ++i)
    if (B->grids[i]->prec != TOMO_FP32 || !z[i] || !dcdz[i]) {
      B->err = "tile autotune: FP32 grids and one z and dcdz array per grid";
      return TOMO_EINVAL;
    }
  if (!B->lockstep || !lockstep_compatible(B->grids)) {
    B->err = "tile autotune: the batch does not run in lockstep";
    return TOMO_EINVAL;
  }
  // candidates: thread rows per CTA x waves of resident CTAs; each timed by the device time
  // of the batched phase (first V-cycle and CG loop, CUDA events on the batch stream) after
  // one untimed call that captures its loop; the median of reps calls
  static const int kRows[] = {8, 4};
  static const int kWaves[] = {2, 4, 8};
  const int ty0 = B->tile_ty, w0 = B->waves;
  std::vector<double> c(n);
  int bi = -1, k = 0;
  double bms = 0.0;
  tomo_status st = TOMO_OK;
  for (int ty : kRows)
    for (int w : kWaves) {
      if (st == TOMO_ECUDA) break;
      tomo_batch_set_tiles(B, ty, w);
      tomo_status sk = batch_lockstep(B, z, c.data(), dcdz, nullptr, nullptr);
      std::vector<double> ms;
      for (int r = 0; r < reps && sk == TOMO_OK; ++r) {
        sk = batch_lockstep(B, z, c.data(), dcdz, nullptr, nullptr);
        ms.push_back(B->phase_ms[1] + B->phase_ms[2]);
      }
      double med = -1.0;
      if (sk == TOMO_OK) {
        std::sort(ms.begin(), ms.end());
        med = ms[ms.size() / 2];
        if (bi < 0 || med < bms) {
          bi = k;
          bms = med;
        }
      } else if (sk == TOMO_ECUDA) {
        st = sk;
      }
      if (res) {
        res[k].tile_rows = ty;
        res[k].waves = w;
        res[k].status = sk;
        res[k].reserved = 0;
        res[k].ms = med;
      }
      ++k;
    }
  if (st == TOMO_OK && bi < 0) {
    st = TOMO_ENOCONV;
    B->err = "tile autotune: no candidate ran";
  }
  if (st != TOMO_OK) {
    tomo_batch_set_tiles(B, ty0, w0);
    return st;
  }
  tomo_batch_set_tiles(B, kRows[bi / 3], kWaves[bi % 3]);
  if (best) *best = bi;
  return TOMO_OK;
}

tomo_status tomo_batch_size(const tomo_batch* B, int32_t* count) {
  if (!B || !count) return TOMO_EINVAL;
  *count = (int32_t)B->grids.size();
  return TOMO_OK;
}

tomo_status tomo_batch_destroy(tomo_batch* B) {
  if (!B) return TOMO_OK;
  for (auto s : B->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (B->bst) {
    cudaStreamSynchronize(B->bst);
    cudaStreamDestroy(B->bst);
  }
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->loop) cudaGraphExecDestroy(B->loop);
  if (B->d_scs) cudaFree(B->d_scs);
  if (B->d_tab) cudaFree(B->d_tab);
  if (B->d_ph) cudaFree(B->d_ph);
  if (B->d_bar) cudaFree(B->d_bar);
  if (B->d_acc) cudaFree(B->d_acc);
  for (auto e : B->wev) cudaEventDestroy(e);
  if (B->bev) cudaEventDestroy(B->bev);
  for (auto e : B->tev)
    if (e) cudaEventDestroy(e);
  delete B;
  return TOMO_OK;
}

const char* tomo_batch_last_error(const tomo_batch* B) {
  if (!B) return g_create_err.c_str();
  return B->err.c_str();
}

const char* tomo_last_error(const tomo_grid* G) {
  if (!G) return g_create_err.c_str();
  return G->err.c_str();
}

}  // extern "C"
