// Shared host-side helpers of the product library: dynamic GF(2) bit vectors,
// the error type that C++ code throws (converted to a tsim_status at the C ABI)
// and exact Z[w] values (w = e^{i pi/4}) used by the host-side evaluator.
#pragma once
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tsim.h"

namespace tsim {

struct Error : std::runtime_error {
  tsim_status code;
  Error(tsim_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(tsim_status c, const std::string& m) { throw Error(c, m); }

// Dense GF(2) vector of fixed length (all vectors of one diagram share it).
struct Bits {
  std::vector<uint64_t> w;
  Bits() = default;
  explicit Bits(size_t nbits) : w((nbits + 63) / 64, 0) {}
  size_t nwords() const { return w.size(); }
  bool get(size_t i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  void set(size_t i) { w[i >> 6] |= 1ull << (i & 63); }
  void reset(size_t i) { w[i >> 6] &= ~(1ull << (i & 63)); }
  void flip(size_t i) { w[i >> 6] ^= 1ull << (i & 63); }
  Bits& operator^=(const Bits& o) {
    if (o.w.size() > w.size()) w.resize(o.w.size(), 0);
    for (size_t i = 0; i < o.w.size(); ++i) w[i] ^= o.w[i];
    return *this;
  }
  bool any() const {
    for (uint64_t x : w)
      if (x) return true;
    return false;
  }
  int first() const {
    for (size_t i = 0; i < w.size(); ++i)
      if (w[i]) return (int)(i * 64 + __builtin_ctzll(w[i]));
    return -1;
  }
  int last() const {
    for (size_t i = w.size(); i-- > 0;)
      if (w[i]) return (int)(i * 64 + 63 - __builtin_clzll(w[i]));
    return -1;
  }
  size_t count() const {
    size_t c = 0;
    for (uint64_t x : w) c += (size_t)__builtin_popcountll(x);
    return c;
  }
  bool operator==(const Bits& o) const {
    size_t n = std::max(w.size(), o.w.size());
    for (size_t i = 0; i < n; ++i) {
      uint64_t a = i < w.size() ? w[i] : 0, b = i < o.w.size() ? o.w[i] : 0;
      if (a != b) return false;
    }
    return true;
  }
  bool operator!=(const Bits& o) const { return !(*this == o); }
  bool operator<(const Bits& o) const {
    size_t n = std::max(w.size(), o.w.size());
    for (size_t i = n; i-- > 0;) {
      uint64_t a = i < w.size() ? w[i] : 0, b = i < o.w.size() ? o.w[i] : 0;
      if (a != b) return a < b;
    }
    return false;
  }
  // parity of (this AND o)
  int dot(const Bits& o) const {
    uint64_t x = 0;
    size_t n = std::min(w.size(), o.w.size());
    for (size_t i = 0; i < n; ++i) x ^= w[i] & o.w[i];
    return __builtin_parityll(x);
  }
  template <class F>
  void for_each(F f) const {
    for (size_t i = 0; i < w.size(); ++i) {
      uint64_t x = w[i];
      while (x) {
        int b = __builtin_ctzll(x);
        f((int)(i * 64 + b));
        x &= x - 1;
      }
    }
  }
};

// Exact element of Z[w] * sqrt2^k: (c0 + c1 w + c2 w^2 + c3 w^3) * sqrt2^k,
// w^4 = -1.  Coefficients are __int128 with overflow checks.
struct ZW {
  __int128 c[4] = {0, 0, 0, 0};
  int k = 0;
  static ZW omega(int j) {
    ZW z;
    j = ((j % 8) + 8) % 8;
    if (j < 4) z.c[j] = 1; else z.c[j - 4] = -1;
    return z;
  }
  bool zero() const { return !(c[0] || c[1] || c[2] || c[3]); }
};

inline __int128 chk_add(__int128 a, __int128 b) {
  __int128 r;
  if (__builtin_add_overflow(a, b, &r)) fail(TSIM_ERR_OVERFLOW_BOUND, "Z[w] overflow");
  return r;
}
inline __int128 chk_mul(__int128 a, __int128 b) {
  __int128 r;
  if (__builtin_mul_overflow(a, b, &r)) fail(TSIM_ERR_OVERFLOW_BOUND, "Z[w] overflow");
  return r;
}
inline ZW zw_mul(const ZW& a, const ZW& b) {
  ZW r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      if (!a.c[i] || !b.c[j]) continue;
      __int128 p = chk_mul(a.c[i], b.c[j]);
      int n = i + j;
      if (n >= 4) r.c[n - 4] = chk_add(r.c[n - 4], -p);
      else r.c[n] = chk_add(r.c[n], p);
    }
  r.k = a.k + b.k;
  return r;
}
inline ZW zw_lower_k(ZW a) {  // same value, exponent k-1: multiply numerator by sqrt2 = w - w^3
  ZW s;
  s.c[1] = 1;
  s.c[3] = -1;
  ZW r = zw_mul(a, s);
  r.k = a.k - 1;
  return r;
}
inline ZW zw_add(ZW a, ZW b) {
  if (a.zero()) return b;
  if (b.zero()) return a;
  while (a.k > b.k) a = zw_lower_k(a);
  while (b.k > a.k) b = zw_lower_k(b);
  ZW r;
  for (int i = 0; i < 4; ++i) r.c[i] = chk_add(a.c[i], b.c[i]);
  r.k = a.k;
  return r;
}

}  // namespace tsim
