// Internal declarations of libtk (host plan layer + kernel launch wrappers).
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tk.h"

namespace tk {

// ------------------------------------------------------------------ symmetry (symbols.cpp)
// Sector algebra of Z2, U(1), SU(2) (Sec. 3.1, Sec. 5.4) and the elementary moves used to
// recouple fusion trees (Sec. 4.2).  All labels use the ABI encoding (SU(2): 2j).
bool sector_valid(int sym, int32_t a);
int32_t sector_unit(int sym);  // label of the trivial sector
int32_t sector_dual(int sym, int32_t a);
int32_t sector_dim(int sym, int32_t a);
void sector_fuse(int sym, int32_t a, int32_t b, std::vector<int32_t>& out);  // ascending
bool sector_nsym(int sym, int32_t a, int32_t b, int32_t c);
double fsymbol(int sym, int32_t a, int32_t b, int32_t c, int32_t d, int32_t e, int32_t f);
double rsymbol(int sym, int32_t a, int32_t b, int32_t c);
double fs_indicator(int sym, int32_t a);  // chi_a
// Coefficient of bending the last leg (label x, space dual flag `was_dual`) off a tree whose
// running label before that leg is u and whose coupled sector is c, onto the last position of
// the opposite tree (new coupled sector u).
double bend_coef(int sym, int32_t x, bool was_dual, int32_t u, int32_t c);

// ------------------------------------------------------------------ structures (structure.cpp)
struct Space {
  int sym = 0;
  std::vector<int32_t> sectors;  // ascending
  std::vector<int64_t> mults;
  bool dual = false;
  std::vector<int32_t> labels;   // tree labels, ascending
  int64_t mult_of_label(int32_t lab) const;
  int64_t dim() const;
  int64_t reduced_dim() const;
  bool same(const Space& o) const {
    return sym == o.sym && dual == o.dual && sectors == o.sectors && mults == o.mults;
  }
  Space flipped() const;
  void finalize();
};

struct Tree {
  std::vector<int32_t> unc;
  std::vector<int32_t> inner;  // running couplings u_2 .. u_{N-1}
  int32_t coupled = 0;
  int64_t size = 1;            // product of leg multiplicities
};

struct Block {
  int32_t c = 0;
  int64_t rows = 0, cols = 0, offset = 0;
  std::vector<int> split, fuse;        // tree ids
  std::vector<int64_t> roff, coff;     // row / column offsets of those trees
};

struct TreePair {
  int block;
  int s, f;                // indices into the block's split / fuse lists
  int64_t offset;          // element offset of the first entry
};

struct Structure {
  int sym = 0;
  std::vector<Space> cod, dom;
  std::vector<Tree> split_trees, fuse_trees;
  std::vector<Block> blocks;
  std::vector<TreePair> pairs;
  std::map<std::vector<int32_t>, std::pair<int, int>> split_pos, fuse_pos;  // key -> (block, idx)
  int64_t numel = 0;
  uint64_t hash = 0;
  int nleg() const { return (int)(cod.size() + dom.size()); }
  int block_of(int32_t c) const;
  // dims of the reduced array of pair p (codomain legs then domain legs)
  void pair_dims(const TreePair& p, std::vector<int64_t>& dims) const;
};

std::vector<int32_t> tree_key(const std::vector<int32_t>& unc, const std::vector<int32_t>& inner,
                              int32_t c);
std::shared_ptr<Structure> build_structure(int sym, const std::vector<Space>& cod,
                                           const std::vector<Space>& dom);

// ------------------------------------------------------------------ plans (plan.cpp)
// One term of Algorithm 10: dst += coef * permute(src).
struct TransformTerm {
  int64_t src_pair, dst_pair;
  double coef;
};

// Device task of the permute kernel (K1): one destination tree pair.
struct PermTask {
  int64_t out_off;       // element offset of the destination reduced array
  int64_t ostr[6];       // destination strides of the merged dims
  int32_t ext[6];        // merged extents
  int32_t irs[6];        // source stride = irs + ics * ld_src
  int32_t ics[6];
  int32_t ndim;
  int32_t mode;          // 0: shared contiguous dim 0; 1: transpose dims (0, tdim); 2: generic;
                         // 3: transpose dims (1, tdim) of vectors along a short dim 0
  int32_t tdim;          // mode 1: the dim that is contiguous in the source; mode 3: the dim
                         // that follows dim 0 in the source
  int32_t src_begin, nsrc;
  int32_t t0, t1;        // tile extents along dim 0 and along the tiled second axis
  int32_t conj;          // 1: conjugate complex values (adjoint)
  int64_t tile_begin;    // first global tile index of this task
};
struct PermSrc {
  int64_t in_off;
  int64_t ld;
  double coef;
};
// One contiguous run of a mode-0 task: dst[e] = sum_k coef_k src_k[ir + e + ic ld_k], e < len.
// Runs of one source with weight 1 carry task = -1 (copy) or -2 (conjugating copy) and the
// absolute source offset in ir: dst[e] = src[ir + e].
struct PermRun {
  int64_t dst, ir, ic;
  int32_t len, task;
};

struct PermutePlan {
  std::shared_ptr<Structure> in, out;
  std::vector<int> perm;      // output leg k <- input leg perm[k]
  bool identity = false;
  std::vector<TransformTerm> terms;   // sorted by destination
  std::vector<PermTask> tasks;    // tile-kernel tasks (transposing / generic)
  std::vector<PermTask> rtasks;   // run-kernel tasks (shared contiguous dim 0)
  std::vector<PermRun> runs;
  std::vector<PermSrc> srcs;
  int64_t total_tiles = 0;
  int32_t run_group = 32;     // lanes per run in the run kernel: 16 when the runs average <= 64 elements
  double bytes = 0;           // algorithmic bytes for one launch (complex counts 16 B/element)
  int dtype = TK_F64;
  // device copies
  PermTask* d_tasks = nullptr;
  PermTask* d_rtasks = nullptr;
  PermRun* d_runs = nullptr;
  PermSrc* d_srcs = nullptr;
  int32_t* d_tile_task = nullptr;  // owning task of every tile
  ~PermutePlan();
};

struct GemmItem {          // one sector GEMM: C~^c (M x N) = A~^c (M x K) * B~^c (K x N)
  int32_t c;
  int64_t M, N, K;
  int64_t a_off, b_off, c_off;
};

struct ZeroItem {
  int64_t off, n;
};

struct ContractPlan {
  std::shared_ptr<PermutePlan> pa, pb, pc;  // pc permutes C~ -> C (null if identity)
  std::shared_ptr<Structure> at, bt, ct, c;
  std::vector<GemmItem> gemms;       // every sector GEMM with K > 0
  std::vector<GemmItem> gemms_fp64;  // run by k_gemm_f64
  std::vector<GemmItem> gemms_oz;    // run by the split-precision tcgen05 kernel
  std::vector<ZeroItem> zeros;
  int gemm_mode = TK_GEMM_FP64;
  int slices = 0;
  int dtype = TK_F64;
  double flops = 0;
  // workspace layout (bytes)
  size_t ws_at = 0, ws_bt = 0, ws_ct = 0, ws_partials = 0, ws_counters = 0, ws_slices = 0, ws_total = 0;
  // device tables
  void* d_gemm_items = nullptr;
  void* d_gemm_tiles = nullptr;
  int64_t n_gemm_tiles = 0;
  // split-K of the FP64 tiles: partial tiles and per-slot arrival counters, both in the caller's
  // workspace; the counters are cleared at the start of every call, so calls of one plan with
  // different workspaces may overlap
  int32_t split_slots = 0;
  size_t partials_bytes = 0;
  void* d_zero = nullptr;
  // split-precision tables (owned; freed by the destructor) and the host-side layout
  std::vector<void*> d_oz;
  int64_t oz_nwork = 0;
  size_t oz_bytes = 0;
  std::shared_ptr<void> oz;
  // work-list choices (0: heuristic); set by the autotuner, applied by finalize_device_tables
  int tune_tile = 0;      // FP64 tiles: 32 or 64 wide
  int tune_split = 0;     // FP64 split-K: 1 off, 2 as many parts as allowed
  int tune_oz_bn = 0;     // split-precision tile width: 64 or 128
  int tune_oz_split = 0;  // split-precision split-K: 1 off, 2 as many parts as allowed
  int tune_oz_img = 0;    // split-precision prep keeps chunks in shared memory: 1 off, 2 on
  size_t ws_base = 0;     // workspace bytes of the permuted operands and C~ (before GEMM scratch)
  // Complex tensors in a split-precision mode: C = A B runs as the four real products
  // Re A Re B, Im A Im B, Re A Im B, Im A Re B of the real plan `re`, on de-interleaved copies of
  // A and B in the workspace; ws_total = ws_cx + re->ws_total.
  std::shared_ptr<ContractPlan> re;
  size_t ws_cx = 0;
  int64_t cx_na = 0, cx_nb = 0, cx_nc = 0;  // element counts of A, B and C
  ~ContractPlan();
};


// Ints after the split-K counters: one out-of-range flag per tile of the double-float rows launch
// (real split-precision plans only; cleared with the counters).
inline int64_t df_guard_words(const ContractPlan& cp) {
  return (cp.gemm_mode != TK_GEMM_FP64 && cp.dtype != TK_C128) ? cp.n_gemm_tiles : 0;
}

// Workspace bytes a call of this contraction plan needs (a complex split-precision plan adds its
// real plan's current size, which the autotuner may change).
inline size_t contract_ws_bytes(const ContractPlan& cp) { return cp.re ? cp.ws_cx + cp.re->ws_total : cp.ws_total; }

struct Ctx;
// (Re)build a contraction plan's device work lists for its current tune_* choices and lay out the
// GEMM part of its workspace.
int finalize_device_tables(Ctx* ctx, ContractPlan& cp);
std::shared_ptr<PermutePlan> make_permute_plan(Ctx* ctx, std::shared_ptr<Structure> in,
                                               const std::vector<int>& p,
                                               const std::vector<int>& q, int dtype);
std::shared_ptr<PermutePlan> make_adjoint_plan(Ctx* ctx, std::shared_ptr<Structure> in, int dtype);
std::shared_ptr<ContractPlan> make_contract_plan(Ctx* ctx, std::shared_ptr<Structure> a,
                                                 const std::vector<int>& pa,
                                                 const std::vector<int>& qa,
                                                 std::shared_ptr<Structure> b,
                                                 const std::vector<int>& pb,
                                                 const std::vector<int>& qb,
                                                 const std::vector<int>& pab,
                                                 const std::vector<int>& qab, int dtype,
                                                 int gemm_mode, int slices);
// output spaces of permute(t, (p, q)) (Algorithm 2)
void permute_spaces(const Structure& s, const std::vector<int>& p, const std::vector<int>& q,
                    std::vector<Space>& cod, std::vector<Space>& dom);

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};

// Device memory of one context: every allocation the library makes (plan tables, the status
// word) goes through the caller's hooks, or cudaMalloc / cudaFree when none were given, and is
// counted.  With a budget set, an allocation or a caller reservation that would take the library
// bytes plus the reserved bytes above it fails with TK_ERR_BUDGET.  Allocations remember their
// DeviceMemory, which therefore lives until its last allocation is freed, after the context.
struct DeviceMemory {
  int device = -1;
  tk_alloc_fn alloc = nullptr;
  tk_free_fn release = nullptr;
  void* user = nullptr;
  std::mutex mu;
  size_t in_use = 0;    // bytes the library holds
  size_t reserved = 0;  // bytes the caller reserved (tk_ctx_reserve)
  size_t budget = 0;    // 0: no budget
  size_t allocations = 0;
};

struct Ctx {
  int device = -1;
  void* stream = nullptr;  // the context's stream: execution calls given a NULL stream use it
  std::shared_ptr<DeviceMemory> mem;
  std::string last_error;
  int64_t launches = 0;
  int num_sms = 0;
  std::mutex mu;
  std::unordered_map<std::string, std::shared_ptr<PermutePlan>> perm_cache;
  std::unordered_map<std::string, std::shared_ptr<ContractPlan>> contract_cache;
  int* d_status = nullptr;  // device status word for bounded waits
  // opt-in kernel profiling: (kernel name, start event, end event) per launch
  bool profiling = false;
  struct Rec {
    const char* name;
    void* start;
    void* end;
  };
  std::vector<Rec> prof;
  // a second stream and two events: in the split-precision modes the CUDA-core products of a
  // contraction run beside its tensor-core chain (fork after the input permutes, join before the
  // output permute); recorded into CUDA graphs as a fork and a join
  void* side = nullptr;
  void* ev_fork = nullptr;
  void* ev_join = nullptr;
  std::mutex side_mu;  // one fork / join at a time: the two events are shared by every caller
};

// ---- block SVD (Algorithm 9 after the two-site step of Algorithm 12)
struct SvdBlock {
  int32_t c;
  int64_t m, n, r;                       // block rows, columns, min(m, n)
  int64_t a_off, u_off, vh_off, s_off;   // element offsets in t, U, V^dagger and the values
};
struct SvdPlan {
  std::shared_ptr<Structure> in, u, vh;  // t : cod <- dom, U : cod <- W, V^dagger : W <- dom
  Space bond;                            // W = sum_c (c, min(rows_c, cols_c))
  std::vector<SvdBlock> blocks;
  int64_t nvalues = 0;                   // singular values, concatenated by sector
  int64_t lwork = 0;                     // doubles of per-block norms / ranks in the workspace
  size_t ws_solver = 0, ws_total = 0;    // bytes of the Jacobi working matrices; whole workspace
  int dtype = TK_F64;
  void* d_jobs = nullptr;                // device job table of the grouped Jacobi launch
  int64_t njobs = 0;
  ~SvdPlan();
};
std::shared_ptr<SvdPlan> make_svd_plan(Ctx* ctx, std::shared_ptr<Structure> in, int dtype);
int run_svd(Ctx* ctx, const SvdPlan& sp, const void* a, void* u, double* s, void* vh, void* ws, void* stream);
int run_svd_truncate(Ctx* ctx, const SvdPlan& sp, const int64_t* keep, const void* u, const double* s, const void* vh,
                     void* ut, double* st, void* vht, void* stream);

// Brackets one launch with events on its stream when the context is profiling.
struct ProfScope {
  Ctx* ctx;
  const char* name;
  void* stream;
  void* start = nullptr;
  ProfScope(Ctx* c, const char* n, void* s);
  ~ProfScope();
};

// ------------------------------------------------------------------ device side (kernels)
// Allocation through the context's DeviceMemory (TK_ERR_BUDGET over budget, TK_ERR_OOM when the
// allocator fails); dev_free finds the allocation's DeviceMemory by address.
int dev_alloc(Ctx* ctx, void** dst, size_t bytes);
int dev_upload(Ctx* ctx, void** dst, const void* src, size_t bytes);
void dev_free(void* p);
bool dev_owns(void* p);  // p is a live allocation of the library (tk_ctx_free checks it)
int launch_permute(Ctx* ctx, const PermutePlan& pp, const void* in, void* out, void* stream);
struct PermJob {
  const PermutePlan* plan;
  const void* in;
  void* out;
};
struct IntClear {
  int* p;
  int64_t n;
  int32_t fill = 0;  // value written to every int (a repeated byte: the no-permute path memsets)
};
// Several permutes in one launch (identity plans are skipped; more than 160 segments take several
// launches), optionally also clearing int arrays (split-K counters) in the same launch.
// zero: optionally, a plan's zero-fill list (blocks with an empty inner dimension) of output c,
// done in the same launch.
struct ZeroJob {
  const ZeroItem* items;  // device
  int64_t nitems, maxn;
  void* c;
  int dtype;  // element type of c (TK_F64 / TK_C128): the launch's type when no permute is left
};
int launch_permutes(Ctx* ctx, const PermJob* jobs, int njobs, void* stream, const IntClear* clears, int nclears,
                    const ZeroJob* zero = nullptr);
int launch_gemm_fp64(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c,
                     void* partials, int* counters, void* stream);
int upload_gemm_tables(Ctx* ctx, ContractPlan& cp);
int launch_gemm_ozaki(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c,
                      void* slices_ws, void* stream);
// The split-precision GEMMs of several requests (their workspaces' slice regions in ws): scaling
// and slicing per request, then one packed tensor-core launch per group of up to 32 requests that
// share mode, tile width and slice count.
int launch_gemm_ozaki_batch(Ctx* ctx, int n, const ContractPlan* const* plans, const void* const* a,
                            const void* const* b, void* const* c, void* const* ws, void* stream);
int upload_ozaki_tables(Ctx* ctx, ContractPlan& cp);
// One-CTA kernel whose bounded mbarrier wait is left to run out (tk_ctx_selftest_timeout).
int launch_wait_selftest(Ctx* ctx, void* stream);
// The launch sequence of one planned contraction with scratch at `ws` (Algorithm 4 / 8).
int run_contract(Ctx* ctx, const ContractPlan& cp, const void* a, const void* b, void* c, void* ws,
                 void* stream);
// Many FP64 contractions with their stages packed into shared launches (tk_contract_batch).
int run_contract_batch(Ctx* ctx, int n, const ContractPlan* const* plans, const void* const* a,
                       const void* const* b, void* const* c, void* const* ws, void* stream);

}  // namespace tk
