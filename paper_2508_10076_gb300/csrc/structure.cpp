// Graded spaces, canonical fusion trees and the block layout of a tensor map.
//
// Block layout (Sec. 3.2 eq. abeliangrouping; Sec. 4.1 canonical splitting trees and the block
// embedding): one column-major block per coupled sector c (ascending), holding the reduced
// arrays of all (splitting tree, fusion tree) pairs with coupled sector c.  Splitting trees
// occupy consecutive row ranges, fusion trees consecutive column ranges, both ordered
// colexicographically (first leg fastest) by uncoupled labels and then by inner labels.  A leg
// of a dual space carries the dual sector as its tree label (Sec. 3.2, transpositions).
#include <algorithm>
#include <functional>

#include "tk_internal.hpp"

namespace tk {

int64_t Space::mult_of_label(int32_t lab) const {
  int32_t a = dual ? sector_dual(sym, lab) : lab;
  auto it = std::lower_bound(sectors.begin(), sectors.end(), a);
  if (it == sectors.end() || *it != a) return 0;
  return mults[it - sectors.begin()];
}

int64_t Space::dim() const {
  int64_t s = 0;
  for (size_t i = 0; i < sectors.size(); ++i) s += mults[i] * sector_dim(sym, sectors[i]);
  return s;
}

int64_t Space::reduced_dim() const {
  int64_t s = 0;
  for (auto m : mults) s += m;
  return s;
}

Space Space::flipped() const {
  Space o = *this;
  o.dual = !dual;
  o.finalize();
  return o;
}

void Space::finalize() {
  labels.clear();
  for (auto a : sectors) labels.push_back(dual ? sector_dual(sym, a) : a);
  std::sort(labels.begin(), labels.end());
}

std::vector<int32_t> tree_key(const std::vector<int32_t>& unc, const std::vector<int32_t>& inner,
                              int32_t c) {
  std::vector<int32_t> k;
  k.reserve(unc.size() + inner.size() + 1);
  k.insert(k.end(), unc.begin(), unc.end());
  k.insert(k.end(), inner.begin(), inner.end());
  k.push_back(c);
  return k;
}

namespace {

void enumerate_trees(int sym, const std::vector<Space>& legs, std::vector<Tree>& out) {
  out.clear();
  const int n = (int)legs.size();
  if (n == 0) {
    Tree t;
    t.coupled = sector_unit(sym);
    t.size = 1;
    out.push_back(t);
    return;
  }
  std::vector<int32_t> unc(n);
  std::vector<int32_t> fz;
  // recursive enumeration of uncoupled labels, then of running couplings
  std::function<void(int)> rec_unc;
  std::function<void(int, int32_t, std::vector<int32_t>&)> rec_inner;
  rec_inner = [&](int k, int32_t u, std::vector<int32_t>& chain) {
    if (k == n) {
      Tree t;
      t.unc = unc;
      t.inner.assign(chain.begin(), chain.end() - (n >= 2 ? 1 : 0));
      t.coupled = n >= 2 ? chain.back() : unc[0];
      t.size = 1;
      for (int i = 0; i < n; ++i) t.size *= legs[i].mult_of_label(unc[i]);
      out.push_back(t);
      return;
    }
    std::vector<int32_t> opts;
    sector_fuse(sym, u, unc[k], opts);
    for (int32_t v : opts) {
      chain.push_back(v);
      rec_inner(k + 1, v, chain);
      chain.pop_back();
    }
  };
  rec_unc = [&](int i) {
    if (i == n) {
      std::vector<int32_t> chain;
      if (n == 1) {
        rec_inner(1, unc[0], chain);
      } else {
        rec_inner(1, unc[0], chain);
      }
      return;
    }
    for (int32_t lab : legs[i].labels) {
      unc[i] = lab;
      rec_unc(i + 1);
    }
  };
  rec_unc(0);
  // colexicographic order: last uncoupled label most significant, then inner labels likewise
  std::stable_sort(out.begin(), out.end(), [](const Tree& x, const Tree& y) {
    for (size_t i = x.unc.size(); i-- > 0;)
      if (x.unc[i] != y.unc[i]) return x.unc[i] < y.unc[i];
    for (size_t i = x.inner.size(); i-- > 0;)
      if (x.inner[i] != y.inner[i]) return x.inner[i] < y.inner[i];
    return false;
  });
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

int Structure::block_of(int32_t c) const {
  int lo = 0, hi = (int)blocks.size();
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (blocks[mid].c < c)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < (int)blocks.size() && blocks[lo].c == c) ? lo : -1;
}

void Structure::pair_dims(const TreePair& p, std::vector<int64_t>& dims) const {
  dims.clear();
  const Block& b = blocks[p.block];
  const Tree& s = split_trees[b.split[p.s]];
  const Tree& f = fuse_trees[b.fuse[p.f]];
  for (size_t i = 0; i < cod.size(); ++i) dims.push_back(cod[i].mult_of_label(s.unc[i]));
  for (size_t i = 0; i < dom.size(); ++i) dims.push_back(dom[i].mult_of_label(f.unc[i]));
}

std::shared_ptr<Structure> build_structure(int sym, const std::vector<Space>& cod,
                                           const std::vector<Space>& dom) {
  auto st = std::make_shared<Structure>();
  st->sym = sym;
  st->cod = cod;
  st->dom = dom;
  for (auto& s : st->cod) s.finalize();
  for (auto& s : st->dom) s.finalize();
  enumerate_trees(sym, st->cod, st->split_trees);
  enumerate_trees(sym, st->dom, st->fuse_trees);
  std::map<int32_t, std::vector<int>> sby, fby;
  for (int i = 0; i < (int)st->split_trees.size(); ++i) sby[st->split_trees[i].coupled].push_back(i);
  for (int i = 0; i < (int)st->fuse_trees.size(); ++i) fby[st->fuse_trees[i].coupled].push_back(i);
  int64_t off = 0;
  for (auto& kv : sby) {
    auto it = fby.find(kv.first);
    if (it == fby.end()) continue;
    Block b;
    b.c = kv.first;
    for (int id : kv.second) {
      b.split.push_back(id);
      b.roff.push_back(b.rows);
      b.rows += st->split_trees[id].size;
    }
    for (int id : it->second) {
      b.fuse.push_back(id);
      b.coff.push_back(b.cols);
      b.cols += st->fuse_trees[id].size;
    }
    if (b.rows == 0 || b.cols == 0) continue;
    b.offset = off;
    off += b.rows * b.cols;
    st->blocks.push_back(b);
  }
  st->numel = off;
  for (int bi = 0; bi < (int)st->blocks.size(); ++bi) {
    const Block& b = st->blocks[bi];
    for (int i = 0; i < (int)b.split.size(); ++i) {
      const Tree& t = st->split_trees[b.split[i]];
      st->split_pos[tree_key(t.unc, t.inner, t.coupled)] = {bi, i};
    }
    for (int j = 0; j < (int)b.fuse.size(); ++j) {
      const Tree& t = st->fuse_trees[b.fuse[j]];
      st->fuse_pos[tree_key(t.unc, t.inner, t.coupled)] = {bi, j};
    }
    for (int i = 0; i < (int)b.split.size(); ++i)
      for (int j = 0; j < (int)b.fuse.size(); ++j)
        st->pairs.push_back(TreePair{bi, i, j, b.offset + b.roff[i] + b.coff[j] * b.rows});
  }
  uint64_t h = 1469598103934665603ull;
  h = mix(h, (uint64_t)sym);
  for (int side = 0; side < 2; ++side) {
    const auto& legs = side == 0 ? st->cod : st->dom;
    h = mix(h, 0xabcdef00ull + side * 7 + legs.size());
    for (const auto& s : legs) {
      h = mix(h, s.dual ? 0x51ull : 0x17ull);
      for (size_t i = 0; i < s.sectors.size(); ++i) {
        h = mix(h, (uint64_t)(uint32_t)s.sectors[i]);
        h = mix(h, (uint64_t)s.mults[i]);
      }
    }
  }
  st->hash = h;
  return st;
}

}  // namespace tk
