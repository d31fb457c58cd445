// Internal host-side declarations of the tomo library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tomo.h"
#include "common.cuh"

namespace tomo {

#ifdef TOMO_CHECKED
// the check words of the translation units with checked kernels (read, then cleared;
// ~0 if the read failed)
unsigned long long check_word_matvec2();
unsigned long long check_word_matvec();
unsigned long long check_word_vec();
unsigned long long check_word_filt();
unsigned long long check_word_vtail();
#endif

// ---------------------------------------------------------------------------------------
// Coarse tail of the V-cycle in one thread-block cluster (vtail.cu): levels [l0, coarsest]
// of one FP32 grid, every pass (element forces, node update, transfers, coarsest solve)
// separated by cluster barriers instead of kernel boundaries.
// ---------------------------------------------------------------------------------------
constexpr int kVtMaxLevels = 8;
constexpr int kVtMaxTailElements = 4096;  // the entry level's elements (about one per thread)
constexpr int kVtMaxDeg = 8;
struct VTailLevel {
  Geom g;
  const float* s;         // element moduli
  const uint8_t* mask;    // fixed-DOF bits per node
  const float* invd;      // D^-1 per node (not for the coarsest)
  float* x;               // iterate (holds the zero-start step on entry when first_done)
  float* xp;              // second smoother buffer
  float* b;               // right-hand side (restricted residual)
  float* t;               // residual
  int K;                  // smoothing degree
  float c1[kVtMaxDeg], c2[kVtMaxDeg];  // Chebyshev coefficients of steps 0..K-1
};
struct VTailArgs {
  int nlev;               // levels of the tail, the last one the dense coarsest
  int first_done;         // the entry level's x already holds the zero-start step
  int nc;                 // coarsest DOFs
  int ld;                 // element-buffer stride (>= the largest level's element count)
  const float* Ainv;      // coarsest: D^-1/2 K^-1 D^-1/2 scaled inverse, row-major
  const float* dsc;       // coarsest: D^-1/2
  float* eb;              // element forces, 24 x ld floats
  const int* skip;        // CG stop flag
  VTailLevel L[kVtMaxLevels];
};
// CTAs of the cluster that runs the tail, 0 if this device cannot launch it
int vtail_ctas();
cudaError_t launch_vtail(cudaStream_t st, const VTailArgs& A, const ElemConst<float>& C);

// Host-side fault injection sites (tomo_inject_fault / TOMO_FAULT); fault_hit(k) is true on
// the armed pass of site k (once per arming).
enum FaultSite {
  FAULT_ALLOC = 0,    // a device allocation of a grid reports TOMO_ENOMEM
  FAULT_SYNC = 1,     // a grid's stream synchronisation reports TOMO_ECUDA (after the real one)
  FAULT_GRAPH = 2,    // a CG-loop graph launch is skipped and reports TOMO_ECUDA
  FAULT_NAN = 3,      // a NaN modulus enters a gradient's material (the solve reports ENAN)
  FAULT_SLOW = 4,     // a served request waits 200 ms on the host before it runs
  FAULT_SITES = 5
};
bool fault_hit(FaultSite k);

// Named host range around a step of the path, visible to NVTX-aware profilers (a no-op
// unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct FilterTap {
  int di, dj, dk;
  double w;
};

void build_unit_stiffness(double nu, double K0[576]);
bool build_hadamard_blocks(const double K0[576], double blk[8][3][3], double* k0diag);
std::vector<FilterTap> filter_taps(double rmin);

// Scalar constants of the four block kinds of K0 in the Hadamard basis (see element.cu).
struct BlockKinds {
  double a0, b0;  // class 0: W = a0 X + b0 (sum X) 1
  double a7, b7;  // class 7: same form
  double ta, tb;  // classes 1, 2, 4: [[ta, tb], [tb, ta]]
  double ua, ud;  // classes 3, 5, 6: ua on the coupled pair (all four entries), ud alone
};
bool block_kinds(const double blk[8][3][3], BlockKinds* out);

// Largest coarsest-level DOF count solved by a dense inverse in one CTA.
constexpr int kMaxDenseDofs = 648;
// Upper bound of lambda_max(D^-1 K) over any grid: max over one element of
// lambda_max(diag(K0)^-1 K0) (x^T K x <= lam_e x^T D x element by element).
constexpr int kTY = 16;  // rows of node columns per CTA in the marching product
// rows per CTA of the batched FP64 residual replacement (256 threads, the CTA size of the
// other batched phases; the per-node result does not depend on the tiling)
constexpr int kRrTY = 8;

enum MarchMode { M_APPLY = 0, M_RESID = 1, M_CHEB = 2 };

template <typename T>
struct MarchArgs {
  Geom g;
  int kz;               // node planes per z-chunk
  const T* s;           // h*E per element
  const uint8_t* mask;  // fixed bits per node
  const T* x;           // input vector (hi part when pair input)
  const T* xlo;         // lo part (pair input) or nullptr
  const T* b;           // right-hand side (RESID, CHEB)
  T* xprev;             // CHEB: x_{k-1} at entry, x_{k+1} at exit (own node only)
  T* y;                 // APPLY / RESID output
  T c1, c2;             // CHEB coefficients
  double* partials;     // dot reduction scratch (APPLY: x.y, CHEB: b.x_new)
  unsigned* counter;
  CgScalars* sc;        // dot result consumer (may be null when no dot)
  int dot_kind;         // 0 none, 1: pq -> alpha, 2: rz_new -> beta
  const int* skip;      // if non-null and *skip != 0 the kernel returns at once
  const CgScalars* gate;  // residual replacement: run only when gate->it % gate->rr_every == 0
  int xprev_zero;       // CHEB: the previous iterate is zero (first step after a zero start)
  // T = double, RESID only: the input is the float pair (xf_hi, xf_lo), joined exactly into
  // double on load, and the residual is written rounded to float into yf
  const float* xf_hi;
  const float* xf_lo;
  float* yf;
  // JOIN RESID only, optional: also the zero-start Jacobi step from the new residual,
  // x1f = c2f * yf * invdf[node] (the finest level's first smoothing step, see k_cg_xr)
  float* x1f;
  const float* invdf;
  float c2f;
};

// Table of a batched FP64 residual launch (gated residual replacement of several FP32
// grids: float-pair input joined in double, residual rounded to float): grid q owns the
// launch's blocks [cta0[q], cta0[q+1]) laid out as its own (gx, gy, z-chunk) grid.
struct MarchRrBatch {
  int n;
  int cta0[kBatchMax + 1];
  short gx[kBatchMax], gy[kBatchMax];
  MarchArgs<double> a[kBatchMax];
};
cudaError_t launch_march_rr_batch(cudaStream_t st, const MarchArgs<double>* a, int n,
                                  const ElemConst<double>& c, int num_sms);

// p[0..n) = v; fT[idx[k]] = f64[idx[k]] = val[k] for k < nnz (vec.cu)
template <typename T>
cudaError_t launch_fill(cudaStream_t st, int64_t n, T* p, T v);
template <typename T>
cudaError_t launch_scatter_load(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                                T* fT, double* f64);
// f^T (u + ulo) over the nonzero load entries (FP64; fixed-order reduction through
// partials/counter); r = scatter of the entries
template <typename T>
cudaError_t launch_sparse_dot(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                              const T* u, const T* ulo, double* partials, unsigned* counter,
                              double* out);
template <typename T>
cudaError_t launch_scatter_vec(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                               T* r);
// one launch: zero the non-null vectors among xhi, xlo, r, p (n each) and set *sc = h
template <typename T>
cudaError_t launch_cg_start(cudaStream_t st, int n, T* xhi, T* xlo, T* r, T* p,
                            tomo::CgScalars* sc, const tomo::CgScalars& h);

// Batched pointwise/vector kernels (vec.cu) for FP32 grids: one entry per grid, the grid
// owning the launch's blocks [cta0[q], cta0[q+1]).
struct JacobiItem {  // zero-start first Chebyshev step x1 = c2 D^-1 b
  Geom g;
  const float* s;
  const uint8_t* mask;
  const float* b;
  float c2, k0diag;
  float* x1;
  const int* skip;
  float* invd;  // optional: D^-1 per node kept for the fused later steps
};
struct RestrictItem {  // r_c = P^T r_f (+ fused zero-start step on the coarse level)
  Geom gf, gc;
  const float* rf;
  float* rc;
  const uint8_t* mask_c;
  const int* skip;
  float* x1;  // nullptr: no fused step
  const float* sc;
  float c2, k0diag;
};
struct ProlongItem {  // x_f += P x_c
  Geom gf, gc;
  const float* xc;
  float* xf;
  const uint8_t* mask_f;
  const int* skip;
};
struct CoarseItem {  // z = D^-1/2 Ainv D^-1/2 r on the coarsest level
  int n;
  const float* Ainv;
  const float* dsc;
  const float* r;
  float* z;
  const int* skip;
};
struct CgXrItem {  // x += alpha p (float pair), r -= alpha q, r.r -> convergence
  int n;
  float* xhi;
  float* xlo;
  float* r;
  const float* p;
  const float* q;
  double* partials;
  unsigned* counter;
  CgScalars* sc;
  float* x1;          // optional: the finest zero-start Jacobi step c2 D^-1 r (see k_cg_xr)
  const float* invd;
  float c2;
};
struct CgPItem {  // p = z + beta p
  int n;
  float* p;
  const float* z;
  CgScalars* sc;
};
template <class Item>
struct FlatBatch {
  int n;
  int cta0[kBatchMax + 1];
  Item a[kBatchMax];
};
cudaError_t launch_jacobi_batch(cudaStream_t st, const JacobiItem* a, int n);
cudaError_t launch_restrict_batch(cudaStream_t st, const RestrictItem* a, int n);
cudaError_t launch_prolong_batch(cudaStream_t st, const ProlongItem* a, int n);
cudaError_t launch_coarse_apply_batch(cudaStream_t st, const CoarseItem* a, int n);
cudaError_t launch_cg_xr_batch(cudaStream_t st, const CgXrItem* a, int n);
cudaError_t launch_cg_p_batch(cudaStream_t st, const CgPItem* a, int n);
// conditional-while control of a batched CG loop: continue while any of the n grids whose
// scalars scs[0..n) (device array) point to has not stopped
cudaError_t launch_loop_cond_batch(cudaStream_t st, cudaGraphConditionalHandle h,
                                   CgScalars* const* scs, int n);

// FP32 two-rows-per-thread product (matvec2.cu); same modes as k_march, no pair input.
struct March2Args {
  Geom g;
  int kz;
  const float* s;
  const uint8_t* mask;
  const float* x;
  const float* b;
  float* xprev;
  float* y;
  float c1, c2;
  double* partials;
  unsigned* counter;
  CgScalars* sc;
  int dot_kind;
  const int* skip;
  int xprev_zero;  // CHEB: the previous iterate is zero (first step after a zero start)
  const float* invd;  // CHEB: D^-1 per node of this level
  // per x-y tile of the launch (32 x 16 node columns with halo): does any node of the
  // tile's columns have a fixed DOF?  nullptr: every tile reads the mask
  const uint8_t* tile_fixed;
};
// Tile flags for k_march2 on a level (see March2Args::tile_fixed), from the host mask.
std::vector<uint8_t> march2_tile_flags(const Geom& g, const std::vector<uint8_t>& hmask);
struct March2Const {
  float a0, b0, a7, b7, ta, tb, ua, ud, k0diag;
};
// Table of a batched k_march2 launch (a kernel parameter): grid q owns the launch's blocks
// [cta0[q], cta0[q+1]) laid out as its own (gx, gy, z-chunk) grid.
struct March2Batch {
  int n;
  int cta0[kBatchMax + 1];
  short gx[kBatchMax], gy[kBatchMax];
  March2Args a[kBatchMax];
};
// The same k_march2 operation on n grids (all with the same mode and dot flag) in
// ceil(n / kBatchMax) launches; each grid gets the tiles of its own launch and z-chunks of
// a[q].kz node planes (kz <= 0: the chunks of its own launch).  Only the fused dot depends
// on the chunking (its per-block partials); the products themselves do not.  ty: thread
// rows per CTA, 8 (the tiles of k_march2) or 4 (tiles of 6 element rows).
cudaError_t launch_march2_batch(cudaStream_t st, int mode, const March2Args* a, int n,
                                const March2Const& c, int num_sms, int ty = 8);
cudaError_t launch_march2(cudaStream_t st, int mode, const March2Args& a, const March2Const& c,
                          int num_sms);

// Persistent lockstep iteration (one cooperative kernel per CG iteration): the batched
// launches of one iteration are recorded instead of launched (kind, unit count and the
// launch's parameter table), then replayed as phases of one kernel, each phase's units
// spread over the co-resident CTAs and the phases separated by grid barriers.
enum PhaseKind : int {
  PH_M2_APPLY = 0, PH_M2_APPLY_DOT, PH_M2_RESID, PH_M2_CHEB, PH_M2_CHEB_DOT, PH_RR,
  PH_JACOBI, PH_RESTRICT, PH_PROLONG, PH_COARSE, PH_CGXR, PH_CGP, PH_COUNT
};
struct PhaseRec {
  int kind;
  int units;
  int join;                          // 1: a further table of the same launch (no barrier)
  std::vector<unsigned char> table;  // the launch's parameter table, bytes
};
// while non-null, the batched launch wrappers append their launch here instead of launching
extern thread_local std::vector<PhaseRec>* g_phase_rec;
template <class Table>
inline void record_phase(int kind, int units, const Table& t, bool cont) {
  PhaseRec r{kind, units, cont ? 1 : 0, std::vector<unsigned char>(sizeof(Table))};
  std::memcpy(r.table.data(), &t, sizeof(Table));
  g_phase_rec->push_back(std::move(r));
}
// Place of one unit (one CTA of the recorded launch) of a phase: grid q of the table, its
// block vb of vnb, and for the products the grid's tile counts gx, gy.
struct UnitDesc {
  int q;
  int vb;
  int vnb;
  short gx, gy;
};
struct DevPhase {
  int kind;
  int units;
  int join;            // no grid barrier before this phase
  int pad;
  long long units_offset;  // of the phase's UnitDesc[units] in the table buffer
  long long offset;  // of the phase's table in the table buffer (256-byte aligned)
};
// Co-resident CTAs of the persistent kernel on this device (occupancy x SMs), 0 if it
// cannot be launched cooperatively.
int persist_ctas(int num_sms, size_t smem);
// One CG iteration of a lockstep batch as one cooperative launch of `ctas` CTAs: phases
// [0, nph) with their tables in `tables`; barrier = two zeroed unsigned words (count,
// generation); a CTA that waits longer than limit_ns at a barrier marks every grid of
// scs[0..nscs) stopped with DEV_TIMEOUT and leaves.  acc (nph + 1 words, may be null):
// acc[p] += the device ns of phase p as CTA 0 sees it, acc[nph] += 1 (adds a barrier after
// the last phase).
cudaError_t launch_persist(cudaStream_t st, const DevPhase* phases, int nph,
                           const unsigned char* tables, const March2Const& k2,
                           const ElemConst<double>& k1, unsigned* barrier, long long limit_ns,
                           CgScalars* const* scs, int nscs, int ctas, size_t smem, unsigned long long* acc);


// All kernels are launched on `st`.  Wrappers return 0 or a cudaError_t.
template <typename T>
cudaError_t launch_march(cudaStream_t st, int mode, const MarchArgs<T>& a, const ElemConst<T>& c,
                         int num_sms, int* grid_ctas);

template <typename T>
cudaError_t launch_jacobi(cudaStream_t st, Geom g, const T* s, const uint8_t* mask, const T* b,
                          T c2, T k0diag, T* x1, T* x0zero, double* partials,
                          unsigned* counter, CgScalars* sc, int dot_kind, const int* skip,
                          T* invd = nullptr);
template <typename T>
cudaError_t launch_restrict(cudaStream_t st, Geom gf, Geom gc, const T* rf, T* rc,
                            const uint8_t* mask_c, const int* skip, T* x1 = nullptr,
                            const T* sc = nullptr, T c2 = T(0), T k0diag = T(0));
template <typename T>
cudaError_t launch_prolong_add(cudaStream_t st, Geom gf, Geom gc, const T* xc, T* xf,
                               const uint8_t* mask_f, const int* skip);
template <typename T>
cudaError_t launch_coarsen_s(cudaStream_t st, Geom gf, Geom gc, const T* sf, T* sc);
// invd[n] = 1 / (k0diag * sum of the node's element moduli), 0 where that is not positive
template <typename T>
cudaError_t launch_invdiag(cudaStream_t st, Geom g, const T* s, T k0diag, T* invd);
template <typename T>
cudaError_t launch_coarse_factor(cudaStream_t st, Geom g, const T* s, const uint8_t* mask,
                                 const DenseK0<T>& K0, T* A, T* dscale, unsigned* status);
template <typename T>
cudaError_t launch_coarse_apply(cudaStream_t st, int n, const T* Ainv, const T* dscale,
                                const T* r, T* z, const int* skip);

// CG recurrences.  xlo != nullptr selects the float-pair iterate (x = xhi + xlo).
template <typename T>
cudaError_t launch_cg_xr(cudaStream_t st, int n, T* xhi, T* xlo, T* r, const T* p, const T* q,
                         double* partials, unsigned* counter, CgScalars* sc, T* x1 = nullptr,
                         const T* invd = nullptr, T c2 = T(0));
template <typename T>
cudaError_t launch_cg_p(cudaStream_t st, int n, T* p, const T* z, CgScalars* sc);
// p = z + beta p with the device-side loop's test in its last block (counter: a zeroed word
// it resets)
template <typename T>
cudaError_t launch_cg_p_cond(cudaStream_t st, int n, T* p, const T* z, CgScalars* sc,
                             cudaGraphConditionalHandle h, unsigned* counter);
int march_blocks_per_sm(int tsize, int mode, bool pair, bool dot);

// Dots and vector helpers.
template <typename TA, typename TB>
cudaError_t launch_dot(cudaStream_t st, int n, const TA* a, const TB* b, const TB* blo,
                       double* partials, unsigned* counter, double* out);
template <typename T>
cudaError_t launch_mask_copy(cudaStream_t st, Geom g, const T* in, const uint8_t* mask, T* out);
// out = in (+ inlo), converted; with a gate, only on residual-replacement iterations.
template <typename TO, typename TI>
cudaError_t launch_convert(cudaStream_t st, int n, const TI* in, const TI* inlo, TO* out,
                           const CgScalars* gate = nullptr);

// Two-scale coarse-graining: z_C = block means of z over N_B^3 element blocks.
template <typename T>
cudaError_t launch_coarse_grain(cudaStream_t st, Geom g, int nb, const T* z, T* zc);

// Filter, material, sensitivity, OC.
template <typename T>
cudaError_t launch_filter(cudaStream_t st, Geom g, const int4* taps, const T* tapw, int ntaps,
                          int radius, const T* in, const T* Hs, T* out, int mode, int material,
                          T E0, T Emin, T penal, T h, T* s_out);
template <typename T>
cudaError_t launch_material(cudaStream_t st, int n, const T* rho, T E0, T Emin, T penal, T h,
                            T* s);
template <typename T>
cudaError_t launch_sensitivity(cudaStream_t st, Geom g, const T* rho, const T* u, const T* ulo,
                               const T* w, const T* wlo, const ElemConst<T>& c, T penal, T E0,
                               T Emin, T h, T* dc);
template <typename T>
cudaError_t launch_oc(cudaStream_t st, int n, const T* z, const T* dc, const T* w, double vmax,
                      double move, T* znew, double* partials, unsigned* counter,
                      double* bracket, double* change_out, int max_blocks);
int oc_partials_needed(int n);
int oc_max_blocks(int n);

}  // namespace tomo

// ------------------------------------------------------------------------------------
// The handle
// ------------------------------------------------------------------------------------
struct tomo_level {
  tomo::Geom g;
  double h;
  void* s = nullptr;        // T[nel]: h * E
  uint8_t* mask = nullptr;  // [nn]
  void* b = nullptr;        // T[3nn] right-hand side (levels >= 1)
  void* x = nullptr;        // T[3nn] iterate
  void* xp = nullptr;       // T[3nn] previous iterate / ping-pong
  void* t = nullptr;        // T[3nn] residual
  uint8_t* tile_fixed = nullptr;  // FP32 grids: k_march2 tiles that hold fixed nodes
  void* invd = nullptr;     // FP32 multigrid levels with a smoother: D^-1 per node
  std::vector<uint8_t> hmask;
};

struct tomo_grid {
  tomo_grid_desc d{};
  int prec = TOMO_FP32;
  size_t tsize = 4;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  tomo::Geom g{};
  std::vector<uint8_t> fixed;  // host copy, 3*nn
  std::vector<double> f;       // host copy, 3*nn
  double K0[576];
  double blk[8][3][3];
  double k0diag = 0.0;
  tomo::BlockKinds kinds{};    // the four block kinds of K0 in the mode basis
  double lam_hi = 0.0;         // Chebyshev upper end
  double cheb_ratio = 10.0;    // Chebyshev interval [lam_hi / ratio, lam_hi]
  std::vector<tomo::FilterTap> taps;
  int4* d_taps = nullptr;      // (di, dj, dk, 0)
  void* d_tapw = nullptr;      // T[ntaps] weights
  int ntaps = 0;
  void* Hs = nullptr;          // T[nel]
  void* dvdz = nullptr;        // T[nel] P^T v (cached)
  bool dvdz_ready = false;     // dvdz holds P^T v (design independent, computed once)
  // the load's nonzero free entries (indices into the 3*nn DOF vector, values)
  int64_t* load_idx = nullptr;
  double* load_val = nullptr;
  int load_nnz = 0;
  std::vector<tomo_level> L;
  int coarse_n = 0;            // coarsest DOFs (dense)
  int filter_radius = 0;       // largest |offset| component of the filter taps
  void* coarseA = nullptr;     // T[n*n]
  void* coarseD = nullptr;     // T[n]
  // fine-level vectors
  void* f_T = nullptr;         // T[3nn] load
  double* f64 = nullptr;       // double[3nn] load (compliance)
  void* r = nullptr;
  void* p = nullptr;
  void* q = nullptr;
  void* xhi = nullptr;         // iterate (FP64: x; FP32: hi part)
  void* xlo = nullptr;         // FP32 only
  void* rho = nullptr;         // T[nel] physical density scratch
  void* dcp = nullptr;         // T[nel] dc/drho scratch
  // reductions
  double* partials = nullptr;
  unsigned* counter = nullptr;
  tomo::CgScalars* sc = nullptr;
  double* dscal = nullptr;     // device doubles for misc results (compliance, change, bracket)
  tomo::CgScalars* h_sc = nullptr;  // pinned
  double* h_scal = nullptr;         // pinned
  // staging for host pointers
  std::vector<void*> stage;
  std::vector<size_t> stage_size;
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  int64_t prof_launches = 0;
  double prof_bytes = 0.0;
  std::vector<int> ev_tag;          // per event pair: -1 fine-level product, else level + 1;
                                    // -2: a launch that found the solve stopped (no work)
  std::vector<double> ev_bytes;     // per event pair: algorithmic bytes of a product launch
  std::vector<int> ev_iter;         // per event pair: CG iteration that enqueued it (0: none)
  std::vector<char> ev_post;        // ... after that iteration's x/r update
  int prof_iter = 0;                // the CG iteration being enqueued (host-issued loop)
  bool prof_post = false;
  double level_ms[16] = {};         // eager V-cycle time per level (all kernels), level 0..15
  int64_t level_n[16] = {};
  size_t dev_bytes = 0;        // device memory held by this grid (cudaMalloc through dalloc)
  bool have_solution = false;
  bool warm_gradient = false;  // tomo_gradient starts CG from the previous solution
  int partials_n = 0;
  double ff = 0.0;                  // ||f||^2 over free DOFs
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  // the coarsest factorisation runs on `side` (high priority) while the first V-cycle's
  // down-sweep runs on `stream`; joined before the first coarsest solve (join_factor)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_factor = nullptr;
  bool factor_pending = false;
  cudaGraphExec_t loop_exec = nullptr;  // device-side PCG loop (conditional while)
  // right-hand side of the next pcg: the load f (rhs_id 0) or an adjoint load (rhs_id 1);
  // each has its own captured loop, since the FP64 residual replacement reads it
  void* rhs_T = nullptr;
  double* rhs64 = nullptr;
  double rhs_ff = 0.0;
  int rhs_id = 0;
  cudaGraphExec_t loop_exec_adj = nullptr;
  void* adj_T = nullptr;       // adjoint load l (masked), T and double
  double* adj64 = nullptr;
  void* adj_hi = nullptr;      // adjoint state lambda (pair on FP32 grids)
  void* adj_lo = nullptr;
  bool use_graph = true;
  // FP32 multigrid grids: the CG x/r update also writes the finest level's zero-start
  // Jacobi step x1 = c2 D^-1 r (D^-1 per node in invd, from the first V-cycle of the solve),
  // so the V-cycles inside the loop skip that launch
  bool fuse_j0 = false;
  // while capturing the device-side loop: the loop's condition handle, set by the last
  // kernel of the iteration (the p update)
  bool cond_capture = false;
  cudaGraphConditionalHandle cond_handle = 0;
  void* invd = nullptr;
  int64_t gen = 0;  // bumped when settings baked into captured loops change (smoother)
  // captured loops (load slot) of smoother settings used before: (fine, coarse, ratio)
  struct CachedLoop {
    int fine, coarse;
    double ratio, lam;
    uint32_t wlevels;
    cudaGraphExec_t exec;
  };
  // bit l: the V-cycle makes two coarse-grid corrections at level l (a W-cycle there)
  uint32_t wlevels = 0;
  // coarse tail in one cluster launch (vtail.cu): entry level (-1: none fits), whether the
  // V-cycle uses it, and its element-force buffer
  int vt_level = -1;
  bool vt_on = false;
  void* vt_eb = nullptr;
  int vt_ld = 0;
  double lam_bound = 0.0;       // the element bound of lambda_max(D^-1 K), always safe
  int64_t bound_fallbacks = 0;  // solves redone at lam_bound after failing at a lower lam_hi
  std::vector<CachedLoop> loop_cache;
  // phase timing (events at phase boundaries; the CG loop stays a graph)
  bool phase_prof = false;
  cudaEvent_t phase_ev[8] = {};
  double phase_ms[8] = {};
  int64_t phase_calls = 0;
  int64_t launches = 0;             // kernels launched (executed graph bodies included)
  int64_t iter_launches = 0;        // kernels in one captured loop body
  // FP64 residual replacement of FP32 grids: r = f - K(x_hi + x_lo) evaluated in FP64
  double* s64 = nullptr;            // h*E at the fine level, double
};
