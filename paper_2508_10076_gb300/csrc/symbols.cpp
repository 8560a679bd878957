// Topological data of Z2, U(1) and SU(2) on the host (Sec. 5.2 and Sec. 5.4).
//
// SU(2) F-symbols follow eq. SU2FSymbol,
//   F^{j1 j2 j3}_{j4}[j5; j6] = sqrt(d5 d6) (-1)^(j1+j2+j3+j4) {j1 j2 j5; j3 j4 j6},
// with the 6j symbol from Racah's formula.  Its square is a rational number; it is evaluated in
// exact big-integer arithmetic and rounded once to the nearest double, so every elementary
// symbol is the correctly rounded value of the exact one.  R^{ab}_c = (-1)^(a+b-c): the plain
// swap of the CG splitting tensor (the sign printed in eq. SU2RSymbol, (-1)^(a+b+c), breaks the
// unit axiom for half-integer c and is read as a misprint).  chi_j = (-1)^(2j).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tk_internal.hpp"

namespace tk {
namespace {

// ---------------------------------------------------------------- minimal unsigned big integer
struct BigU {
  std::vector<uint32_t> d;  // little-endian limbs, no leading zeros
  BigU() {}
  explicit BigU(uint64_t v) {
    while (v) {
      d.push_back((uint32_t)v);
      v >>= 32;
    }
  }
  bool zero() const { return d.empty(); }
  void trim() {
    while (!d.empty() && d.back() == 0) d.pop_back();
  }
  int bits() const {
    if (d.empty()) return 0;
    int b = 32 * (int)(d.size() - 1);
    uint32_t t = d.back();
    while (t) {
      ++b;
      t >>= 1;
    }
    return b;
  }
  bool bit(int i) const {
    size_t w = (size_t)i / 32;
    return w < d.size() && ((d[w] >> (i % 32)) & 1u);
  }
};

int cmp(const BigU& a, const BigU& b) {
  if (a.d.size() != b.d.size()) return a.d.size() < b.d.size() ? -1 : 1;
  for (size_t i = a.d.size(); i-- > 0;)
    if (a.d[i] != b.d[i]) return a.d[i] < b.d[i] ? -1 : 1;
  return 0;
}

BigU add(const BigU& a, const BigU& b) {
  BigU r;
  size_t n = std::max(a.d.size(), b.d.size());
  r.d.resize(n + 1);
  uint64_t carry = 0;
  for (size_t i = 0; i < n; ++i) {
    uint64_t s = carry;
    if (i < a.d.size()) s += a.d[i];
    if (i < b.d.size()) s += b.d[i];
    r.d[i] = (uint32_t)s;
    carry = s >> 32;
  }
  r.d[n] = (uint32_t)carry;
  r.trim();
  return r;
}

BigU sub(const BigU& a, const BigU& b) {  // requires a >= b
  BigU r;
  r.d.resize(a.d.size());
  int64_t borrow = 0;
  for (size_t i = 0; i < a.d.size(); ++i) {
    int64_t s = (int64_t)a.d[i] - borrow - (i < b.d.size() ? (int64_t)b.d[i] : 0);
    borrow = s < 0;
    if (s < 0) s += (int64_t)1 << 32;
    r.d[i] = (uint32_t)s;
  }
  r.trim();
  return r;
}

BigU mul(const BigU& a, const BigU& b) {
  if (a.zero() || b.zero()) return BigU();
  BigU r;
  r.d.assign(a.d.size() + b.d.size(), 0);
  for (size_t i = 0; i < a.d.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.d.size(); ++j) {
      uint64_t t = (uint64_t)a.d[i] * b.d[j] + r.d[i + j] + carry;
      r.d[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    size_t k = i + b.d.size();
    while (carry) {
      uint64_t t = (uint64_t)r.d[k] + carry;
      r.d[k] = (uint32_t)t;
      carry = t >> 32;
      ++k;
    }
  }
  r.trim();
  return r;
}

BigU shl(const BigU& a, int s) {
  if (a.zero() || s == 0) return a;
  BigU r;
  int w = s / 32, b = s % 32;
  r.d.assign(a.d.size() + w + 1, 0);
  for (size_t i = 0; i < a.d.size(); ++i) {
    uint64_t v = (uint64_t)a.d[i] << b;
    r.d[i + w] |= (uint32_t)v;
    r.d[i + w + 1] |= (uint32_t)(v >> 32);
  }
  r.trim();
  return r;
}

// quotient of a / b (b != 0) by binary long division
BigU divq(const BigU& a, const BigU& b) {
  BigU q, r;
  int nb = a.bits();
  q.d.assign((nb + 31) / 32 + 1, 0);
  for (int i = nb - 1; i >= 0; --i) {
    r = shl(r, 1);
    if (a.bit(i)) {
      if (r.d.empty()) r.d.push_back(0);
      r.d[0] |= 1u;
    }
    if (cmp(r, b) >= 0) {
      r = sub(r, b);
      q.d[i / 32] |= 1u << (i % 32);
    }
  }
  q.trim();
  return q;
}

// floor(sqrt(n)) for n < 2^128 (digit-by-digit on unsigned __int128)
uint64_t isqrt128(unsigned __int128 n) {
  unsigned __int128 res = 0, bit = (unsigned __int128)1 << 126;
  while (bit > n) bit >>= 2;
  while (bit) {
    if (n >= res + bit) {
      n -= res + bit;
      res = (res >> 1) + bit;
    } else {
      res >>= 1;
    }
    bit >>= 2;
  }
  return (uint64_t)res;
}

unsigned __int128 to128(const BigU& a) {
  unsigned __int128 v = 0;
  for (size_t i = a.d.size(); i-- > 0;) v = (v << 32) | a.d[i];
  return v;
}

// Correctly rounded (nearest-even) double of sqrt(num / den), num, den > 0.
double sqrt_ratio(const BigU& num, const BigU& den) {
  // choose 2k so that Q = num * 4^k / den has about 120 bits (then r = isqrt(Q) ~ 60 bits)
  int e = num.bits() - den.bits();
  int twok = 120 - e;
  if (twok & 1) ++twok;
  BigU n2 = num, d2 = den;
  if (twok >= 0)
    n2 = shl(num, twok);
  else
    d2 = shl(den, -twok);
  BigU Q = divq(n2, d2);
  unsigned __int128 q = to128(Q);  // < 2^122 by construction
  uint64_t r = isqrt128(q);
  // exact iff r^2 * d2 == n2
  BigU rr = mul(BigU(r), BigU(r));
  bool exact = cmp(mul(rr, d2), n2) == 0;
  int nb = 64 - __builtin_clzll(r);
  int sh = nb - 53;
  uint64_t mant = r;
  int exp2 = -twok / 2;
  if (sh > 0) {
    uint64_t rem = r & ((1ull << sh) - 1);
    uint64_t half = 1ull << (sh - 1);
    mant = r >> sh;
    bool up = rem > half || (rem == half && (!exact || (mant & 1)));
    if (up) ++mant;
    exp2 += sh;
  }
  return std::ldexp((double)mant, exp2);
}

uint64_t fact_small(int n) {  // only used for n <= 20
  uint64_t f = 1;
  for (int i = 2; i <= n; ++i) f *= (uint64_t)i;
  return f;
}

BigU fact(int n) {
  if (n <= 20) return BigU(fact_small(n));
  BigU f(fact_small(20));
  for (int i = 21; i <= n; ++i) f = mul(f, BigU((uint64_t)i));
  return f;
}

struct Frac {  // non-negative rational
  BigU n, d;
};

Frac frac_add(const Frac& a, const Frac& b) {
  if (a.n.zero()) return b;
  if (b.n.zero()) return a;
  return Frac{add(mul(a.n, b.d), mul(b.n, a.d)), mul(a.d, b.d)};
}

bool tri2(int a, int b, int c) {  // triangle rule on 2j labels
  return std::abs(a - b) <= c && c <= a + b && ((a + b + c) % 2 == 0);
}

// F^{j1 j2 j3}_{j4}[j5; j6] for SU(2), labels 2j; exact then rounded once.
double su2_fsymbol_exact(int t1, int t2, int t3, int t4, int t5, int t6) {
  // 6j {a b c; d e f} = {j1 j2 j5; j3 j4 j6}
  const int a = t1, b = t2, c = t5, d = t3, e = t4, f = t6;
  if (!tri2(a, b, c) || !tri2(a, e, f) || !tri2(d, b, f) || !tri2(d, e, c)) return 0.0;
  const int tri[4][3] = {{a, b, c}, {a, e, f}, {d, b, f}, {d, e, c}};
  // prefactor squared: product of Delta^2 = (x+y-z)!(x-y+z)!(-x+y+z)!/(x+y+z+1)!
  BigU pn(1), pd(1);
  int al[4];
  for (int i = 0; i < 4; ++i) {
    int x = tri[i][0], y = tri[i][1], z = tri[i][2];
    pn = mul(pn, mul(fact((x + y - z) / 2), mul(fact((x - y + z) / 2), fact((-x + y + z) / 2))));
    pd = mul(pd, fact((x + y + z) / 2 + 1));
    al[i] = (x + y + z) / 2;
  }
  int be[3] = {(a + b + d + e) / 2, (b + c + e + f) / 2, (c + a + f + d) / 2};
  int tmin = *std::max_element(al, al + 4), tmax = *std::min_element(be, be + 3);
  Frac pos{BigU(), BigU(1)}, neg{BigU(), BigU(1)};
  for (int t = tmin; t <= tmax; ++t) {
    BigU den(1);
    for (int i = 0; i < 4; ++i) den = mul(den, fact(t - al[i]));
    for (int i = 0; i < 3; ++i) den = mul(den, fact(be[i] - t));
    Frac term{fact(t + 1), den};
    if (t % 2 == 0)
      pos = frac_add(pos, term);
    else
      neg = frac_add(neg, term);
  }
  // S = pos - neg
  BigU lhs = mul(pos.n, neg.d), rhs = mul(neg.n, pos.d);
  int sgn = cmp(lhs, rhs);
  if (sgn == 0) return 0.0;
  BigU sn = sgn > 0 ? sub(lhs, rhs) : sub(rhs, lhs);
  BigU sd = mul(pos.d, neg.d);
  // F^2 = d5 d6 * pre^2 * S^2
  BigU num = mul(mul(BigU((uint64_t)(t5 + 1) * (uint64_t)(t6 + 1)), pn), mul(sn, sn));
  BigU den = mul(pd, mul(sd, sd));
  double v = sqrt_ratio(num, den);
  int phase = (t1 + t2 + t3 + t4) / 2;
  if (phase & 1) sgn = -sgn;
  return sgn > 0 ? v : -v;
}

std::mutex g_fmu;
std::unordered_map<uint64_t, double> g_fcache;

}  // namespace

// Deligne products S1 x S2 (Sec. 5.2 product sectors): a sector is the pair (a1, a2), encoded as
// a1 * 4096 + field(a2) with field(a2) = a2 + 2048 for a U(1) second factor (|a2| < 2048) and
// a2 otherwise, so that the integer order is the lexicographic order of the pairs.  Fusion,
// duals and dimensions act factor by factor; F, R, the Frobenius-Schur indicator and the bend
// coefficient of a product are the products of the factors' values.
namespace {
constexpr int32_t kPairShift = 4096, kU1Offset = 2048;
bool product_sym(int sym, int& s1, int& s2) {
  switch (sym) {
    case TK_SYM_U1_SU2: s1 = TK_SYM_U1; s2 = TK_SYM_SU2; return true;
    case TK_SYM_Z2_U1: s1 = TK_SYM_Z2; s2 = TK_SYM_U1; return true;
  }
  return false;
}
void split_pair(int s2, int32_t a, int32_t& a1, int32_t& a2) {
  a1 = (a >= 0 ? a : a - (kPairShift - 1)) / kPairShift;  // floor division
  const int32_t f = a - a1 * kPairShift;
  a2 = s2 == TK_SYM_U1 ? f - kU1Offset : f;
}
int32_t join_pair(int s2, int32_t a1, int32_t a2) { return a1 * kPairShift + (s2 == TK_SYM_U1 ? a2 + kU1Offset : a2); }
}  // namespace

int32_t sector_unit(int sym) {
  int s1, s2;
  return product_sym(sym, s1, s2) ? join_pair(s2, 0, 0) : 0;
}

bool sector_valid(int sym, int32_t a) {
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2;
    split_pair(s2, a, a1, a2);
    return sector_valid(s1, a1) && sector_valid(s2, a2) && a1 > -(1 << 18) && a1 < (1 << 18);
  }
  switch (sym) {
    case TK_SYM_Z2: return a == 0 || a == 1;
    case TK_SYM_U1: return true;
    case TK_SYM_SU2: return a >= 0 && a <= 4095;
  }
  return false;
}

int32_t sector_dual(int sym, int32_t a) {
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2;
    split_pair(s2, a, a1, a2);
    return join_pair(s2, sector_dual(s1, a1), sector_dual(s2, a2));
  }
  return sym == TK_SYM_U1 ? -a : a;
}

int32_t sector_dim(int sym, int32_t a) {
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2;
    split_pair(s2, a, a1, a2);
    return sector_dim(s1, a1) * sector_dim(s2, a2);
  }
  return sym == TK_SYM_SU2 ? a + 1 : 1;
}

void sector_fuse(int sym, int32_t a, int32_t b, std::vector<int32_t>& out) {
  out.clear();
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2, b1, b2;
    split_pair(s2, a, a1, a2);
    split_pair(s2, b, b1, b2);
    std::vector<int32_t> c1, c2;
    sector_fuse(s1, a1, b1, c1);
    sector_fuse(s2, a2, b2, c2);
    for (int32_t x : c1)
      for (int32_t y : c2) out.push_back(join_pair(s2, x, y));  // ascending: x major, y minor
    return;
  }
  switch (sym) {
    case TK_SYM_Z2: out.push_back(a ^ b); break;
    case TK_SYM_U1: out.push_back(a + b); break;
    case TK_SYM_SU2:
      for (int32_t c = std::abs(a - b); c <= a + b; c += 2) out.push_back(c);
      break;
  }
}

bool sector_nsym(int sym, int32_t a, int32_t b, int32_t c) {
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2, b1, b2, c1, c2;
    split_pair(s2, a, a1, a2);
    split_pair(s2, b, b1, b2);
    split_pair(s2, c, c1, c2);
    return sector_nsym(s1, a1, b1, c1) && sector_nsym(s2, a2, b2, c2);
  }
  switch (sym) {
    case TK_SYM_Z2: return c == (a ^ b);
    case TK_SYM_U1: return c == a + b;
    case TK_SYM_SU2: return tri2(a, b, c);
  }
  return false;
}

double fsymbol(int sym, int32_t a, int32_t b, int32_t c, int32_t d, int32_t e, int32_t f) {
  if (!sector_nsym(sym, a, b, e) || !sector_nsym(sym, e, c, d) || !sector_nsym(sym, b, c, f) ||
      !sector_nsym(sym, a, f, d))
    return 0.0;
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t x1[6], x2[6];
    const int32_t x[6] = {a, b, c, d, e, f};
    for (int i = 0; i < 6; ++i) split_pair(s2, x[i], x1[i], x2[i]);
    return fsymbol(s1, x1[0], x1[1], x1[2], x1[3], x1[4], x1[5]) *
           fsymbol(s2, x2[0], x2[1], x2[2], x2[3], x2[4], x2[5]);
  }
  if (sym != TK_SYM_SU2) return 1.0;
  if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0 || f < 0 || a > 1023 || b > 1023 || c > 1023 ||
      d > 1023 || e > 1023 || f > 1023)
    return 0.0;
  uint64_t key = ((uint64_t)a) | ((uint64_t)b << 10) | ((uint64_t)c << 20) | ((uint64_t)d << 30) |
                 ((uint64_t)e << 40) | ((uint64_t)f << 50);
  {
    std::lock_guard<std::mutex> lk(g_fmu);
    auto it = g_fcache.find(key);
    if (it != g_fcache.end()) return it->second;
  }
  double v = su2_fsymbol_exact(a, b, c, d, e, f);
  std::lock_guard<std::mutex> lk(g_fmu);
  g_fcache[key] = v;
  return v;
}

double rsymbol(int sym, int32_t a, int32_t b, int32_t c) {
  if (!sector_nsym(sym, a, b, c)) return 0.0;
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2, b1, b2, c1, c2;
    split_pair(s2, a, a1, a2);
    split_pair(s2, b, b1, b2);
    split_pair(s2, c, c1, c2);
    return rsymbol(s1, a1, b1, c1) * rsymbol(s2, a2, b2, c2);
  }
  if (sym != TK_SYM_SU2) return 1.0;
  return (((a + b - c) / 2) & 1) ? -1.0 : 1.0;
}

double fs_indicator(int sym, int32_t a) {
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t a1, a2;
    split_pair(s2, a, a1, a2);
    return fs_indicator(s1, a1) * fs_indicator(s2, a2);
  }
  if (sym != TK_SYM_SU2) return 1.0;
  return (a & 1) ? -1.0 : 1.0;
}

double bend_coef(int sym, int32_t x, bool was_dual, int32_t u, int32_t c) {
  // Overlap of the bent tree pair with the canonical one, divided by its norm d_u:
  //   (was_dual ? 1 : chi_x) * (-1)^(x + c - u) * sqrt(d_c / d_u)
  // (for SU(2); abelian symmetries give 1; a product multiplies its factors' values).
  int s1, s2;
  if (product_sym(sym, s1, s2)) {
    int32_t x1, x2, u1, u2, c1, c2;
    split_pair(s2, x, x1, x2);
    split_pair(s2, u, u1, u2);
    split_pair(s2, c, c1, c2);
    return bend_coef(s1, x1, was_dual, u1, c1) * bend_coef(s2, x2, was_dual, u2, c2);
  }
  if (sym != TK_SYM_SU2) return 1.0;
  double s = was_dual ? 1.0 : fs_indicator(sym, x);
  if (((x + c - u) / 2) & 1) s = -s;
  if (c == u) return s;
  return s * std::sqrt((double)(c + 1) / (double)(u + 1));
}

}  // namespace tk

extern "C" double tk_fsymbol(int sym, int32_t a, int32_t b, int32_t c, int32_t d, int32_t e,
                             int32_t f) {
  if (sym < 0 || sym > TK_SYM_Z2_U1) return 0.0;
  for (int32_t x : {a, b, c, d, e, f})
    if (!tk::sector_valid(sym, x)) return 0.0;
  return tk::fsymbol(sym, a, b, c, d, e, f);
}

extern "C" double tk_rsymbol(int sym, int32_t a, int32_t b, int32_t c) {
  if (sym < 0 || sym > TK_SYM_Z2_U1) return 0.0;
  for (int32_t x : {a, b, c})
    if (!tk::sector_valid(sym, x)) return 0.0;
  return tk::rsymbol(sym, a, b, c);
}
