// Structure-only planning: permute transforms (Algorithm 10 via local moves, Sec. 4.2), the
// permute kernel's task tables, and contraction plans (Algorithm 4 / Algorithm 8).
//
// A permute(t, (p, q)) is resolved per input fusion-tree pair as in Sec. 4.2 ("bend everything
// to the splitting side, swap adjacent legs, bend back"):
//   1. bend the domain legs, last first, onto the end of the splitting tree (right bends);
//   2. sort the splitting legs into the order (p..., reversed q...) by adjacent swaps (bubble
//      sort, Sec. 2.2 footnote), each swap an R-move on the first vertex or an F-R-F sequence
//      elsewhere;
//   3. bend the last N2' splitting legs back onto the fusion tree.
// Every step maps a canonical tree pair to a sparse combination of canonical tree pairs; the
// composition gives the coefficients of Algorithm 10.  For abelian symmetries every
// coefficient is 1 and each channel maps to exactly one channel (Algorithm 6).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>
#include <stdexcept>

#include "tk_internal.hpp"

namespace tk {

namespace {

// ---------------------------------------------------------------- tree-pair label algebra
struct TP {
  std::vector<int32_t> su, si;  // splitting tree: uncoupled and inner labels
  int32_t c = 0;
  std::vector<int32_t> fu, fi;  // fusion tree
};

std::vector<int32_t> encode(const TP& t) {
  std::vector<int32_t> k;
  k.reserve(t.su.size() + t.si.size() + 1 + t.fu.size() + t.fi.size() + 2);
  k.push_back((int32_t)t.su.size());
  k.push_back((int32_t)t.fu.size());
  k.insert(k.end(), t.su.begin(), t.su.end());
  k.insert(k.end(), t.si.begin(), t.si.end());
  k.push_back(t.c);
  k.insert(k.end(), t.fu.begin(), t.fu.end());
  k.insert(k.end(), t.fi.begin(), t.fi.end());
  return k;
}

TP decode(const std::vector<int32_t>& k) {
  TP t;
  size_t n1 = (size_t)k[0], n2 = (size_t)k[1];
  size_t i = 2;
  t.su.assign(k.begin() + i, k.begin() + i + n1);
  i += n1;
  size_t ni1 = n1 >= 2 ? n1 - 2 : 0;
  t.si.assign(k.begin() + i, k.begin() + i + ni1);
  i += ni1;
  t.c = k[i++];
  t.fu.assign(k.begin() + i, k.begin() + i + n2);
  i += n2;
  size_t ni2 = n2 >= 2 ? n2 - 2 : 0;
  t.fi.assign(k.begin() + i, k.begin() + i + ni2);
  return t;
}

using Vec = std::map<std::vector<int32_t>, double>;

// running label before the last leg of a tree with uncoupled `u` and inner `in`
int32_t before_last(int sym, const std::vector<int32_t>& u, const std::vector<int32_t>& in) {
  size_t n = u.size();
  if (n == 1) return sector_unit(sym);
  if (n == 2) return u[0];
  return in[n - 3];
}

// last fusion leg -> last splitting leg
Vec bend_f2s(int sym, const Vec& v, bool was_dual) {
  Vec out;
  for (const auto& kv : v) {
    TP t = decode(kv.first);
    int32_t b = t.fu.back();
    int32_t u = before_last(sym, t.fu, t.fi);
    double coef = bend_coef(sym, b, was_dual, u, t.c);
    TP n;
    n.su = t.su;
    n.su.push_back(sector_dual(sym, b));
    n.si = t.si;
    if (t.su.size() >= 2) n.si.push_back(t.c);
    n.c = u;
    n.fu.assign(t.fu.begin(), t.fu.end() - 1);
    if (t.fu.size() >= 3) n.fi.assign(t.fi.begin(), t.fi.end() - 1);
    out[encode(n)] += kv.second * coef;
  }
  return out;
}

// last splitting leg -> last fusion leg
Vec bend_s2f(int sym, const Vec& v, bool was_dual) {
  Vec out;
  for (const auto& kv : v) {
    TP t = decode(kv.first);
    int32_t a = t.su.back();
    int32_t u = before_last(sym, t.su, t.si);
    double coef = bend_coef(sym, a, was_dual, u, t.c);
    TP n;
    n.fu = t.fu;
    n.fu.push_back(sector_dual(sym, a));
    n.fi = t.fi;
    if (t.fu.size() >= 2) n.fi.push_back(t.c);
    n.c = u;
    n.su.assign(t.su.begin(), t.su.end() - 1);
    if (t.su.size() >= 3) n.si.assign(t.si.begin(), t.si.end() - 1);
    out[encode(n)] += kv.second * coef;
  }
  return out;
}

// swap splitting legs k and k+1
Vec swap_legs(int sym, const Vec& v, int k) {
  Vec out;
  std::vector<int32_t> opts, fopts;
  for (const auto& kv : v) {
    TP t = decode(kv.first);
    const int n = (int)t.su.size();
    if (k == 0) {
      int32_t r1 = (n == 2) ? t.c : t.si[0];
      double coef = rsymbol(sym, t.su[0], t.su[1], r1);
      TP m = t;
      std::swap(m.su[0], m.su[1]);
      out[encode(m)] += kv.second * coef;
      continue;
    }
    int32_t u = (k == 1) ? t.su[0] : t.si[k - 2];
    int32_t e = t.si[k - 1];
    int32_t d = (k + 1 == n - 1) ? t.c : t.si[k];
    int32_t a = t.su[k], b = t.su[k + 1];
    sector_fuse(sym, u, b, opts);
    sector_fuse(sym, a, b, fopts);
    for (int32_t e2 : opts) {
      if (!sector_nsym(sym, e2, a, d)) continue;
      double coef = 0.0;
      for (int32_t f : fopts) {
        if (!sector_nsym(sym, u, f, d)) continue;
        coef += fsymbol(sym, u, a, b, d, e, f) * rsymbol(sym, a, b, f) *
                fsymbol(sym, u, b, a, d, e2, f);
      }
      if (coef == 0.0) continue;
      TP m = t;
      std::swap(m.su[k], m.su[k + 1]);
      m.si[k - 1] = e2;
      out[encode(m)] += kv.second * coef;
    }
  }
  return out;
}

// Coefficients below this magnitude are exact zeros of the recoupling algebra that survive as
// rounding residue of F-R-F sums; genuine SU(2) coefficients of the label ranges handled here
// are many orders of magnitude larger.
constexpr double kDropTol = 1e-13;

int64_t prod64(const std::vector<int64_t>& v, size_t b, size_t e) {
  int64_t p = 1;
  for (size_t i = b; i < e; ++i) p *= v[i];
  return p;
}

std::string perm_key(uint64_t h, const std::vector<int>& p, const std::vector<int>& q, int dtype) {
  std::ostringstream os;
  os << h << "|" << dtype << "|";
  for (int x : p) os << x << ",";
  os << ";";
  for (int x : q) os << x << ",";
  return os.str();
}

}  // namespace

void permute_spaces(const Structure& s, const std::vector<int>& p, const std::vector<int>& q,
                    std::vector<Space>& cod, std::vector<Space>& dom) {
  const int n1 = (int)s.cod.size();
  cod.clear();
  dom.clear();
  for (int i : p) cod.push_back(i < n1 ? s.cod[i] : s.dom[i - n1].flipped());
  for (int j : q) dom.push_back(j < n1 ? s.cod[j].flipped() : s.dom[j - n1]);
}

static void build_transform(PermutePlan& pp, const std::vector<int>& p, const std::vector<int>& q) {
  const Structure& in = *pp.in;
  const Structure& out = *pp.out;
  const int sym = in.sym;
  const int n1 = (int)in.cod.size(), n2 = (int)in.dom.size(), n = n1 + n2;
  std::vector<int> target(p.begin(), p.end());
  for (size_t j = q.size(); j-- > 0;) target.push_back(q[j]);
  std::vector<int> pos(n);
  for (int j = 0; j < n; ++j) pos[target[j]] = j;
  // pair index of output pairs: block -> first pair id
  std::vector<int64_t> out_start(out.blocks.size() + 1, 0);
  for (size_t b = 0; b < out.blocks.size(); ++b)
    out_start[b + 1] = out_start[b] + (int64_t)out.blocks[b].split.size() * out.blocks[b].fuse.size();

  pp.terms.clear();
  for (int64_t pi = 0; pi < (int64_t)in.pairs.size(); ++pi) {
    const TreePair& pr = in.pairs[pi];
    const Block& blk = in.blocks[pr.block];
    const Tree& s = in.split_trees[blk.split[pr.s]];
    const Tree& f = in.fuse_trees[blk.fuse[pr.f]];
    TP t;
    t.su = s.unc;
    t.si = s.inner;
    t.c = blk.c;
    t.fu = f.unc;
    t.fi = f.inner;
    Vec v;
    v[encode(t)] = 1.0;
    std::vector<int> legs_s, legs_f;
    std::vector<char> dual(n);
    for (int i = 0; i < n1; ++i) {
      legs_s.push_back(i);
      dual[i] = in.cod[i].dual;
    }
    for (int j = 0; j < n2; ++j) {
      legs_f.push_back(n1 + j);
      dual[n1 + j] = in.dom[j].dual;
    }
    // 1. bend all domain legs onto the splitting tree
    while (!legs_f.empty()) {
      int leg = legs_f.back();
      v = bend_f2s(sym, v, dual[leg]);
      dual[leg] = !dual[leg];
      legs_f.pop_back();
      legs_s.push_back(leg);
    }
    // 2. bubble sort by adjacent swaps
    for (int pass = 0; pass < n; ++pass) {
      bool moved = false;
      for (int k = 0; k + 1 < n; ++k) {
        if (pos[legs_s[k]] > pos[legs_s[k + 1]]) {
          v = swap_legs(sym, v, k);
          std::swap(legs_s[k], legs_s[k + 1]);
          moved = true;
        }
      }
      if (!moved) break;
    }
    // 3. bend back the domain legs
    for (size_t j = 0; j < q.size(); ++j) {
      int leg = legs_s.back();
      v = bend_s2f(sym, v, dual[leg]);
      dual[leg] = !dual[leg];
      legs_s.pop_back();
      legs_f.push_back(leg);
    }
    for (const auto& kv : v) {
      if (std::fabs(kv.second) <= kDropTol) continue;
      TP o = decode(kv.first);
      auto is = out.split_pos.find(tree_key(o.su, o.si, o.c));
      auto jf = out.fuse_pos.find(tree_key(o.fu, o.fi, o.c));
      if (is == out.split_pos.end() || jf == out.fuse_pos.end() || is->second.first != jf->second.first)
        throw std::runtime_error("permute transform produced a tree pair outside the output structure");
      int b = is->second.first;
      int64_t dst = out_start[b] + (int64_t)is->second.second * out.blocks[b].fuse.size() + jf->second.second;
      pp.terms.push_back(TransformTerm{pi, dst, kv.second});
    }
  }
  std::stable_sort(pp.terms.begin(), pp.terms.end(),
                   [](const TransformTerm& a, const TransformTerm& b) { return a.dst_pair < b.dst_pair; });
}

// Longest run handled by one warp visit; longer contiguous runs are split.  Runs shorter than
// kMinRun would leave most of a warp idle: such tasks take the element-wise tile path instead.
constexpr int64_t kRunChunk = 1024;
constexpr int32_t kMinRun = 8;

// One destination task from its merged dims: run tasks (mode 0, contiguous on both sides) become
// runs; the rest go to the tile kernel as transposes (mode 1) or element-wise (mode 2).
static void emit_task(PermutePlan& pp, PermTask t, std::vector<int64_t>& ext, std::vector<int64_t>& ostr,
                      std::vector<int64_t>& irs, std::vector<int64_t>& ics, double& bytes) {
  const double esize = pp.dtype == TK_C128 ? 16.0 : 8.0;
  if (ext.empty()) {
    ext.push_back(1);
    ostr.push_back(1);
    irs.push_back(1);
    ics.push_back(0);
  }
  if (ext.size() > 6) throw std::runtime_error("permute task with more than 6 non-mergeable dims");
  {
    int64_t elems = 1;
    for (int64_t x : ext) elems *= x;
    if (elems >= ((int64_t)1 << 31)) throw std::runtime_error("permute task with 2^31 or more elements");
  }
  t.ndim = (int32_t)ext.size();
  int64_t total = 1;
  for (size_t k = 0; k < ext.size(); ++k) {
    t.ext[k] = (int32_t)ext[k];
    t.ostr[k] = ostr[k];
    t.irs[k] = (int32_t)irs[k];
    t.ics[k] = (int32_t)ics[k];
    total *= ext[k];
  }
  int tdim = -1;
  for (int k = 1; k < t.ndim; ++k)
    if (t.irs[k] == 1 && t.ics[k] == 0) tdim = k;
  bytes += esize * (double)total * (1.0 + (double)t.nsrc);
  if (t.ostr[0] == 1 && t.irs[0] == 1 && t.ics[0] == 0 && t.ext[0] >= kMinRun) {
    // mode 0: contiguous runs along dim 0 on both sides -> one run per outer position
    t.mode = 0;
    const int32_t task_id = (int32_t)pp.rtasks.size();
    pp.rtasks.push_back(t);
    const PermSrc s0 = pp.srcs[(size_t)t.src_begin];
    const bool plain = t.nsrc == 1 && s0.coef == 1.0;  // a copy (conjugating for adjoint tasks)
    const int64_t outer = total / t.ext[0];
    for (int64_t o = 0; o < outer; ++o) {
      int64_t rem = o, dst = t.out_off, ir = 0, ic = 0;
      for (int k = 1; k < t.ndim; ++k) {
        const int64_t x = rem % t.ext[k];
        rem /= t.ext[k];
        dst += x * t.ostr[k];
        ir += x * t.irs[k];
        ic += x * t.ics[k];
      }
      for (int64_t e0 = 0; e0 < t.ext[0]; e0 += kRunChunk) {
        const int32_t len = (int32_t)std::min<int64_t>(kRunChunk, t.ext[0] - e0);
        if (plain)  // the source offset resolved here: the kernel makes no table lookups
          pp.runs.push_back(PermRun{dst + e0, s0.in_off + ir + e0 + ic * s0.ld, 0, len, t.conj ? -2 : -1});
        else
          pp.runs.push_back(PermRun{dst + e0, ir + e0, ic, len, task_id});
      }
    }
    return;
  }
  // a short leading dim (2..4 elements, e.g. an MPO leg) contiguous on both sides, followed by
  // dim 1 in the destination and by some dim vd in the source: transpose vectors of that length
  int vd = -1;
  if (t.ndim >= 3 && t.ostr[0] == 1 && t.irs[0] == 1 && t.ics[0] == 0 && t.ext[0] >= 2 && t.ext[0] <= 4 &&
      t.ostr[1] == t.ext[0])
    for (int k = 2; k < t.ndim; ++k)
      if (t.irs[k] == t.ext[0] && t.ics[k] == 0) vd = k;
  if (t.ostr[0] == 1 && tdim > 0 && t.ext[0] >= 4 && t.ext[tdim] >= 4) {
    t.mode = 1;
    t.tdim = tdim;
    t.t0 = 32;
    t.t1 = 32;
  } else if (vd > 0) {
    t.mode = 3;
    t.tdim = vd;
    t.t0 = 16;
    t.t1 = 16;
  } else {
    t.mode = 2;
  }
  pp.tasks.push_back(t);
}

// A permute with few, long runs leaves the run kernel short of warps (one group of lanes per
// run, each with about 1 KB of loads in flight): cut the runs into pieces of at least 128
// elements until there are about kRunTarget of them (one and a half per warp slot of a 152-SM
// part with four resident 8-warp blocks per SM).  A piece of a run is again a run: both sides
// stay contiguous, and the source index advances with the destination (plain runs carry a
// resolved source offset, gathering runs an in-task index).
constexpr int64_t kRunTarget = 152 * 4 * 8 * 3 / 2;
constexpr int64_t kRunPieceMin = 128;
static void balance_runs(PermutePlan& pp) {
  const int64_t n = (int64_t)pp.runs.size();
  if (n == 0 || n >= kRunTarget) return;
  int64_t elems = 0;
  for (const PermRun& r : pp.runs) elems += r.len;
  int64_t piece = (elems + kRunTarget - 1) / kRunTarget;
  piece = std::max<int64_t>(kRunPieceMin, (piece + 31) / 32 * 32);
  if (piece >= kRunChunk) return;
  std::vector<PermRun> out;
  out.reserve((size_t)(elems / piece + n));
  for (const PermRun& r : pp.runs)
    for (int32_t e0 = 0; e0 < r.len; e0 += (int32_t)piece)
      out.push_back(PermRun{r.dst + e0, r.ir + e0, r.ic, (int32_t)std::min<int64_t>(piece, r.len - e0), r.task});
  pp.runs.swap(out);
}

// Tile prefix of the tile-kernel tasks; lanes per run of the run kernel.
static void finish_tiles(PermutePlan& pp) {
  balance_runs(pp);
  if (!pp.runs.empty()) {
    int64_t elems = 0;
    for (const PermRun& r : pp.runs) elems += r.len;
    pp.run_group = elems <= 64 * (int64_t)pp.runs.size() ? 16 : 32;  // short runs: two per warp
  }
  int64_t acc = 0;
  for (auto& t : pp.tasks) {
    t.tile_begin = acc;
    int64_t total = 1;
    for (int k = 0; k < t.ndim; ++k) total *= t.ext[k];
    if (t.mode == 1) {
      int64_t outer = total / ((int64_t)t.ext[0] * t.ext[t.tdim]);
      acc += ((t.ext[0] + 31) / 32) * (int64_t)((t.ext[t.tdim] + 31) / 32) * outer;
    } else if (t.mode == 3) {
      int64_t outer = total / ((int64_t)t.ext[0] * t.ext[1] * t.ext[t.tdim]);
      acc += ((t.ext[1] + 15) / 16) * (int64_t)((t.ext[t.tdim] + 15) / 16) * outer;
    } else {
      acc += (total + 255) / 256;
    }
  }
  pp.total_tiles = acc;
}

static void build_tasks(PermutePlan& pp) {
  const Structure& in = *pp.in;
  const Structure& out = *pp.out;
  const int n = out.nleg();
  const int n1o = (int)out.cod.size(), n1i = (int)in.cod.size();
  std::vector<int> inv(n);
  for (int k = 0; k < n; ++k) inv[pp.perm[k]] = k;
  pp.tasks.clear();
  pp.rtasks.clear();
  pp.runs.clear();
  pp.srcs.clear();
  double bytes = 0;
  std::vector<int64_t> od, idims;
  size_t ti = 0;
  for (int64_t y = 0; y < (int64_t)out.pairs.size(); ++y) {
    const TreePair& op = out.pairs[y];
    const Block& ob = out.blocks[op.block];
    out.pair_dims(op, od);
    PermTask t;
    std::memset(&t, 0, sizeof(t));
    t.out_off = op.offset;
    t.src_begin = (int32_t)pp.srcs.size();
    while (ti < pp.terms.size() && pp.terms[ti].dst_pair == y) {
      const TransformTerm& tt = pp.terms[ti];
      const TreePair& ip = in.pairs[tt.src_pair];
      pp.srcs.push_back(PermSrc{ip.offset, in.blocks[ip.block].rows, tt.coef});
      ++ti;
    }
    t.nsrc = (int32_t)pp.srcs.size() - t.src_begin;
    // When every source block has the same leading dimension ld (always so for one source), a
    // column step is a fixed element stride ld: fold it into the row stride, so that contiguity
    // along a domain leg (e.g. blocks with one row) is seen by the mode choice below.
    int64_t fold = pp.srcs[t.src_begin].ld;
    for (int32_t q = t.src_begin + 1; q < t.src_begin + t.nsrc; ++q)
      if (pp.srcs[q].ld != fold) fold = 0;
    // strides per output leg
    idims.assign(n, 1);
    for (int k = 0; k < n; ++k) idims[pp.perm[k]] = od[k];
    std::vector<int64_t> ext, ostr, irs, ics;
    for (int k = 0; k < n; ++k) {
      if (od[k] == 1) continue;
      int64_t os = k < n1o ? prod64(od, 0, k) : ob.rows * prod64(od, n1o, k);
      int j = pp.perm[k];
      int64_t r = 0, c = 0;
      if (j < n1i)
        r = prod64(idims, 0, j);
      else if (fold > 0)
        r = prod64(idims, n1i, j) * fold;
      else
        c = prod64(idims, n1i, j);
      // merge with the previous kept dim when contiguous on both sides
      if (!ext.empty()) {
        size_t m = ext.size() - 1;
        if (ostr[m] * ext[m] == os && irs[m] * ext[m] == r && ics[m] * ext[m] == c) {
          ext[m] *= od[k];
          continue;
        }
      }
      ext.push_back(od[k]);
      ostr.push_back(os);
      irs.push_back(r);
      ics.push_back(c);
    }
    if (ext.empty()) {
      ext.push_back(1);
      ostr.push_back(1);
      irs.push_back(1);
      ics.push_back(0);
    }
    emit_task(pp, t, ext, ostr, irs, ics, bytes);
  }

  finish_tiles(pp);
  pp.bytes = bytes;
}

static void upload_permute_tables(Ctx* ctx, PermutePlan& pp) {
  if (!ctx || ctx->device < 0 || (pp.tasks.empty() && pp.runs.empty())) return;
  std::vector<int32_t> owner((size_t)pp.total_tiles);
  for (size_t i = 0; i < pp.tasks.size(); ++i) {
    const int64_t end = i + 1 < pp.tasks.size() ? pp.tasks[i + 1].tile_begin : pp.total_tiles;
    for (int64_t k = pp.tasks[i].tile_begin; k < end; ++k) owner[(size_t)k] = (int32_t)i;
  }
  int rc = TK_OK;
  if (!pp.tasks.empty()) {
    rc = dev_upload(ctx, (void**)&pp.d_tasks, pp.tasks.data(), pp.tasks.size() * sizeof(PermTask));
    if (rc == TK_OK && !owner.empty())
      rc = dev_upload(ctx, (void**)&pp.d_tile_task, owner.data(), owner.size() * sizeof(int32_t));
  }
  if (rc == TK_OK && !pp.rtasks.empty())
    rc = dev_upload(ctx, (void**)&pp.d_rtasks, pp.rtasks.data(), pp.rtasks.size() * sizeof(PermTask));
  if (rc == TK_OK && !pp.runs.empty())
    rc = dev_upload(ctx, (void**)&pp.d_runs, pp.runs.data(), pp.runs.size() * sizeof(PermRun));
  if (rc == TK_OK && !pp.srcs.empty())
    rc = dev_upload(ctx, (void**)&pp.d_srcs, pp.srcs.data(), pp.srcs.size() * sizeof(PermSrc));
  if (rc != TK_OK) throw Error{rc, "uploading permute tables failed"};
}

// Adjoint t^dagger : dom <- cod of t : cod <- dom.  With orthonormal canonical trees the splitting
// and fusion trees exchange roles, so block c of the result is the conjugate transpose of block c
// of t: one transpose task per block on the permute kernels (conjugation for complex data).
std::shared_ptr<PermutePlan> make_adjoint_plan(Ctx* ctx, std::shared_ptr<Structure> in, int dtype) {
  std::string key = "adj#" + perm_key(in->hash, {}, {}, dtype);
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->perm_cache.find(key);
    if (it != ctx->perm_cache.end()) return it->second;
  }
  auto pp = std::make_shared<PermutePlan>();
  pp->in = in;
  pp->dtype = dtype;
  pp->out = build_structure(in->sym, in->dom, in->cod);
  pp->identity = false;
  const Structure& out = *pp->out;
  double bytes = 0;
  for (const Block& ob : out.blocks) {
    const int ib = in->block_of(ob.c);
    if (ib < 0) throw Error{TK_ERR_ARG, "adjoint: coupled sector missing from the input"};
    const Block& bl = in->blocks[ib];  // rows x cols; the result block is cols x rows
    PermTask t;
    std::memset(&t, 0, sizeof(t));
    t.out_off = ob.offset;
    t.src_begin = (int32_t)pp->srcs.size();
    t.nsrc = 1;
    t.conj = dtype == TK_C128 ? 1 : 0;
    pp->srcs.push_back(PermSrc{bl.offset, bl.rows, 1.0});
    // result (k, r) <- input (r, k): dim 0 runs over the input's columns (source stride rows),
    // dim 1 over its rows (source stride 1); extents of 1 are dropped
    std::vector<int64_t> ext, ostr, irs, ics;
    if (bl.cols > 1) {
      ext.push_back(bl.cols);
      ostr.push_back(1);
      irs.push_back(bl.rows);
      ics.push_back(0);
    }
    if (bl.rows > 1) {
      ext.push_back(bl.rows);
      ostr.push_back(bl.cols);
      irs.push_back(1);
      ics.push_back(0);
    }
    emit_task(*pp, t, ext, ostr, irs, ics, bytes);
  }
  finish_tiles(*pp);
  pp->bytes = bytes;
  upload_permute_tables(ctx, *pp);
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->perm_cache[key] = pp;
  }
  return pp;
}

std::shared_ptr<PermutePlan> make_permute_plan(Ctx* ctx, std::shared_ptr<Structure> in,
                                               const std::vector<int>& p,
                                               const std::vector<int>& q, int dtype) {
  const int n = in->nleg();
  std::vector<int> all(p);
  all.insert(all.end(), q.begin(), q.end());
  std::vector<int> chk(all);
  std::sort(chk.begin(), chk.end());
  for (int i = 0; i < n; ++i)
    if ((int)chk.size() != n || chk[i] != i) throw Error{TK_ERR_PERM, "(p, q) is not a permutation of the legs"};
  if (n == 0) throw Error{TK_ERR_PERM, "empty permutation"};
  std::string key = perm_key(in->hash, p, q, dtype);
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->perm_cache.find(key);
    if (it != ctx->perm_cache.end()) return it->second;
  }
  auto pp = std::make_shared<PermutePlan>();
  pp->in = in;
  pp->dtype = dtype;
  pp->perm = all;
  std::vector<Space> cod, dom;
  permute_spaces(*in, p, q, cod, dom);
  pp->out = build_structure(in->sym, cod, dom);
  pp->identity = (int)p.size() == (int)in->cod.size();
  for (int i = 0; i < n && pp->identity; ++i) pp->identity = all[i] == i;
  build_transform(*pp, p, q);
  build_tasks(*pp);
  upload_permute_tables(ctx, *pp);
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->perm_cache[key] = pp;
  }
  return pp;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Smallest M, N and K of a sector product that runs on the split-precision tensor-core kernel.
constexpr int64_t kSplitMinK = 16, kRowsMaxN = 8, kRowsMaxK = 64;

int finalize_device_tables(Ctx* ctx, ContractPlan& cp) {
  for (void* p : {cp.d_gemm_items, cp.d_gemm_tiles, cp.d_zero}) dev_free(p);
  cp.d_gemm_items = cp.d_gemm_tiles = cp.d_zero = nullptr;
  for (void* p : cp.d_oz) dev_free(p);
  cp.d_oz.clear();
  cp.oz.reset();
  cp.partials_bytes = 0;
  cp.split_slots = 0;
  int rc = upload_gemm_tables(ctx, cp);
  if (rc != TK_OK) return rc;
  size_t off = cp.ws_base;
  cp.ws_partials = off;
  off += align256(cp.partials_bytes);
  cp.ws_counters = off;
  off += align256((size_t)(cp.split_slots + df_guard_words(cp)) * sizeof(int));
  cp.ws_slices = off;
  cp.ws_total = off;
  if (cp.gemm_mode != TK_GEMM_FP64) {
    if ((rc = upload_ozaki_tables(ctx, cp)) != TK_OK) return rc;
    cp.ws_total = cp.ws_slices + align256(cp.oz_bytes);
  }
  return TK_OK;
}

std::shared_ptr<ContractPlan> make_contract_plan(Ctx* ctx, std::shared_ptr<Structure> a,
                                                 const std::vector<int>& pa,
                                                 const std::vector<int>& qa,
                                                 std::shared_ptr<Structure> b,
                                                 const std::vector<int>& pb,
                                                 const std::vector<int>& qb,
                                                 const std::vector<int>& pab,
                                                 const std::vector<int>& qab, int dtype,
                                                 int gemm_mode, int slices) {
  if (a->sym != b->sym) throw Error{TK_ERR_SPACE_MISMATCH, "A and B have different symmetries"};
  if (dtype == TK_C128 && gemm_mode != TK_GEMM_FP64) {
    // complex operands, split-precision products: four real products of the real plan (the
    // recoupling coefficients are real, so permutes act on real and imaginary parts alike)
    auto re = make_contract_plan(ctx, a, pa, qa, b, pb, qb, pab, qab, TK_F64, gemm_mode, slices);
    auto cp = std::make_shared<ContractPlan>();
    cp->dtype = TK_C128;
    cp->gemm_mode = gemm_mode;
    cp->slices = slices;
    cp->re = re;
    cp->pa = re->pa;
    cp->pb = re->pb;
    cp->pc = re->pc;
    cp->at = re->at;
    cp->bt = re->bt;
    cp->ct = re->ct;
    cp->c = re->c;
    cp->gemms = re->gemms;
    cp->flops = 4.0 * re->flops;  // 8 MKN
    cp->cx_na = a->numel;
    cp->cx_nb = b->numel;
    cp->cx_nc = re->c->numel;
    cp->ws_cx = 2 * align256((size_t)cp->cx_na * 8) + 2 * align256((size_t)cp->cx_nb * 8) +
                4 * align256((size_t)cp->cx_nc * 8);
    cp->ws_total = cp->ws_cx + re->ws_total;
    return cp;
  }
  std::ostringstream os;
  os << perm_key(a->hash, pa, qa, dtype) << "#" << perm_key(b->hash, pb, qb, dtype) << "#";
  for (int x : pab) os << x << ",";
  os << ";";
  for (int x : qab) os << x << ",";
  os << "#" << gemm_mode << "#" << slices;
  std::string key = os.str();
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->contract_cache.find(key);
    if (it != ctx->contract_cache.end()) return it->second;
  }
  auto cp = std::make_shared<ContractPlan>();
  cp->dtype = dtype;
  cp->gemm_mode = gemm_mode;
  cp->slices = slices;
  cp->pa = make_permute_plan(ctx, a, pa, qa, dtype);
  cp->pb = make_permute_plan(ctx, b, pb, qb, dtype);
  cp->at = cp->pa->out;
  cp->bt = cp->pb->out;
  const Structure& at = *cp->at;
  const Structure& bt = *cp->bt;
  if (at.dom.size() != bt.cod.size()) throw Error{TK_ERR_SPACE_MISMATCH, "domain(A~) and codomain(B~) differ in length"};
  for (size_t i = 0; i < at.dom.size(); ++i)
    if (!at.dom[i].same(bt.cod[i]))
      throw Error{TK_ERR_SPACE_MISMATCH, "domain(A~) != codomain(B~) (spaces or duality differ)"};
  cp->ct = build_structure(at.sym, at.cod, bt.dom);
  const Structure& ct = *cp->ct;
  // sector GEMMs (Algorithm 8): C~^c = A~^c B~^c, zero block when K_c = 0
  const double fl = dtype == TK_C128 ? 8.0 : 2.0;
  for (const Block& cb : ct.blocks) {
    int ia = at.block_of(cb.c), ib = bt.block_of(cb.c);
    if (ia < 0 || ib < 0) {
      cp->zeros.push_back(ZeroItem{cb.offset, cb.rows * cb.cols});
      continue;
    }
    const Block& ab = at.blocks[ia];
    const Block& bb = bt.blocks[ib];
    if (ab.rows != cb.rows || bb.cols != cb.cols || ab.cols != bb.rows)
      throw Error{TK_ERR_SPACE_MISMATCH, "inconsistent block shapes"};
    cp->gemms.push_back(GemmItem{cb.c, cb.rows, cb.cols, ab.cols, ab.offset, bb.offset, cb.offset});
    cp->flops += fl * (double)cb.rows * (double)cb.cols * (double)ab.cols;
  }
  // output permute
  std::vector<int> all(pab);
  all.insert(all.end(), qab.begin(), qab.end());
  bool ident = (int)pab.size() == (int)ct.cod.size() && (int)all.size() == ct.nleg();
  for (size_t i = 0; i < all.size() && ident; ++i) ident = all[i] == (int)i;
  if (!ident) {
    cp->pc = make_permute_plan(ctx, cp->ct, pab, qab, dtype);
    cp->c = cp->pc->out;
  } else {
    if ((int)all.size() != ct.nleg()) throw Error{TK_ERR_PERM, "(pab, qab) is not a permutation"};
    cp->c = cp->ct;
  }
  const size_t es = dtype == TK_C128 ? 16 : 8;
  size_t off = 0;
  if (!cp->pa->identity) {
    cp->ws_at = off;
    off += align256(at.numel * es);
  }
  if (!cp->pb->identity) {
    cp->ws_bt = off;
    off += align256(bt.numel * es);
  }
  if (cp->pc) {
    cp->ws_ct = off;
    off += align256(ct.numel * es);
  }
  // Engine per sector product in the split-precision modes.  The tensor path pads M to 128, N to a
  // multiple of 16 and K to 32, but runs ~100x the FP64 rate, so it takes every product except
  // very shallow ones (K < 16) and the skinny matrix-product-operator steps (N <= 8 with K below
  // 64, e.g. K = N = 4), which are memory-bound and stay on the CUDA cores (double-float row
  // kernel).  A product with N <= 8 but a deep K goes to the tensor path: the row kernel walks K
  // serially per row.
  for (const GemmItem& g : cp->gemms) {
    const bool thin = g.K < kSplitMinK || (g.N <= kRowsMaxN && g.K < kRowsMaxK);
    if (gemm_mode == TK_GEMM_FP64 || thin)
      cp->gemms_fp64.push_back(g);
    else
      cp->gemms_oz.push_back(g);
  }
  cp->ws_base = off;
  cp->ws_slices = off;
  cp->ws_total = off;
  if (ctx && ctx->device >= 0) {
    int rc = finalize_device_tables(ctx, *cp);
    if (rc != TK_OK) throw Error{rc, "uploading GEMM tables failed"};
  } else if (gemm_mode != TK_GEMM_FP64) {
    cp->ws_total = cp->ws_slices;  // sized on device contexts only
  }
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->contract_cache[key] = cp;
  }
  return cp;
}

}  // namespace tk
