// Host side of the GB300 sampler: packing a compiled program into one
// read-only device blob (channels, noise groups, outputs, marginal tables in
// their device layouts), uploading it, the per-device status word, batch
// plans (persistent launches, autotuning, CUDA graphs), the debug dump of
// table values, and sampling without device allocation.  The kernels live in
// kernels.cuh, instantiated per X width in kern_w*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <unordered_map>

#include "device.h"
#include "devtypes.h"
#include "zx.h"

namespace tsim {

#define TSIM_CUDA(x)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) fail(TSIM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

constexpr int kMaxDevices = 64;

// Status word of each device (bits ST_*), allocated on the first upload to
// that device and read (then cleared) by tsim_sync.
std::mutex g_status_mu;
int* g_status_dev[kMaxDevices];

int* status_word(int dev) {
  if (dev < 0 || dev >= kMaxDevices) fail(TSIM_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!g_status_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, 256);
    if (e != cudaSuccess) fail(TSIM_ERR_OOM, std::string("cudaMalloc of the status word: ") + cudaGetErrorString(e));
    e = cudaMemset(p, 0, 256);
    if (e != cudaSuccess) {
      cudaFree(p);
      fail(TSIM_ERR_CUDA, std::string("cudaMemset of the status word: ") + cudaGetErrorString(e));
    }
    g_status_dev[dev] = (int*)p;
  }
  return g_status_dev[dev];
}

// ---- sampling without device allocation.  Some callers cannot call
// cudaMalloc: code running inside a memory pool or allocator it does not
// own, real-time loops that must not touch the driver's allocator, or hosts
// whose device memory is carved up ahead of time.  For them the program's
// device tables -- the scratch that tsim_sample allocates once per program --
// and a status word live in the fixed array below (kNoAllocBytes, 4 MiB;
// every GPU that loads the library holds it until the process exits): the
// status word in its first kNoAllocHead bytes, the tables after it.
constexpr size_t kNoAllocBytes = (size_t)4 << 20;
constexpr size_t kNoAllocHead = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
// device address of g_noalloc_scratch per device, from cudaGetSymbolAddress
// (the host-side name of the array is not a device address)
void* g_noalloc_dev[kMaxDevices];

}  // namespace

struct DeviceProgram {
  DevView v{};
  void* blob = nullptr;
  int device = -1;
};

void device_release(DeviceProgram* d) {
  if (!d) return;
  if (d->blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (d->device >= 0 && d->device != cur) cudaSetDevice(d->device);
    cudaFree(d->blob);
    if (d->device >= 0 && d->device != cur) cudaSetDevice(cur);
  }
  delete d;
}

bool monomial_of(const ZW& v, int* zero, int* s, int* j) {
  if (v.zero()) { *zero = 1; *s = 0; *j = 0; return true; }
  *zero = 0;
  // strip common factors 2 = sqrt2^2; a monomial then has the coefficient
  // pattern of w^j (one entry +-1) or of sqrt2 w^j = w^(j+1) - w^(j+3)
  // (entries +-1 two places apart)
  __int128 c[4] = {v.c[0], v.c[1], v.c[2], v.c[3]};
  int k = v.k;
  while (!(c[0] & 1) && !(c[1] & 1) && !(c[2] & 1) && !(c[3] & 1)) {
    for (auto& x : c) x /= 2;
    k += 2;
  }
  int nz = 0;
  for (auto x : c) nz += x != 0;
  for (int jj = 0; jj < 8; ++jj) {
    ZW m1 = ZW::omega(jj);
    if (nz == 1 && m1.c[0] == c[0] && m1.c[1] == c[1] && m1.c[2] == c[2] && m1.c[3] == c[3]) {
      *s = k;
      *j = jj;
      return true;
    }
    ZW a = ZW::omega(jj + 1), b = ZW::omega(jj + 3);
    bool eq = nz == 2;
    for (int i = 0; i < 4 && eq; ++i) eq = (a.c[i] - b.c[i]) == c[i];
    if (eq) {
      *s = k + 1;
      *j = jj;
      return true;
    }
  }
  return false;
}

// ------------------------------------------------------ host-side packing
namespace {

int padded_words_or_zero(int W) {
  for (int p : {1, 2, 4, 8, 16, 32})
    if (W <= p) return p;
  return 0;
}

struct Packer {
  std::vector<unsigned char> b;
  size_t section() {
    b.resize((b.size() + 255) & ~(size_t)255, 0);
    return b.size();
  }
  void put(const void* p, size_t n) {
    size_t o = b.size();
    b.resize(o + n);
    if (n) std::memcpy(b.data() + o, p, n);
  }
  void put_padded(const std::vector<uint64_t>& m, int W) {
    for (int i = 0; i < W; ++i) {
      uint64_t x = (size_t)i < m.size() ? m[(size_t)i] : 0;
      put(&x, 8);
    }
  }
};

// Four packed increments of one factor, inc = j | s << 11 | zero << 21
// (J in bits 0-10, S in 11-20, vanishing factors in 21-31), s relative to the
// factor's smallest magnitude exponent smin.
bool factor_lut(int kind, int alpha, int beta, uint32_t inc[4], int* smin_out, int* spread) {
  Factor fc;
  fc.kind = kind;
  fc.alpha = alpha;
  fc.beta = beta;
  int zs[4], ss[4], js[4], smin = 1 << 20, smax = -(1 << 20);
  for (int idx = 0; idx < 4; ++idx) {
    if (!monomial_of(factor_value(fc, idx & 1, idx >> 1), &zs[idx], &ss[idx], &js[idx])) return false;
    if (!zs[idx]) { smin = std::min(smin, ss[idx]); smax = std::max(smax, ss[idx]); }
  }
  if (smin > smax) smin = smax = 0;
  if (smax - smin > 3) return false;
  for (int idx = 0; idx < 4; ++idx)
    inc[idx] = zs[idx] ? (1u << 21) : ((uint32_t)js[idx] | ((uint32_t)(ss[idx] - smin) << 11));
  *smin_out = smin;
  *spread = smax - smin;
  return true;
}

int log2_ceil(unsigned __int128 x) {
  int l = 0;
  while (l < 127 && ((unsigned __int128)1 << l) < x) ++l;
  return l;
}

struct PackError {
  tsim_status st;
  const char* msg;
};

struct Lut {
  uint32_t inc[4];
  int smin, spread;
};

struct FacKey {
  int kind, alpha, beta, ia, ib;
  double t = 0;  // arbitrary-angle factors: the angle
  bool operator<(const FacKey& o) const {
    return std::tie(kind, alpha, beta, ia, ib, t) < std::tie(o.kind, o.alpha, o.beta, o.ia, o.ib, o.t);
  }
};

// A term of a sliced table: constant phase j, magnitude exponent d, and the
// parity indices of each operation code (sorted); dead terms vanish for
// every shot.
struct SlTerm {
  int d = 0, j = 0;
  bool dead = false;
  std::vector<uint64_t> ops[kSlCodes];  // parity indices (qa | qb << 32 for pi-pairs)
};

// How one factor acts on (J, Z): J += j00 + da a + db b + dab ab (mod 8) on
// the (a, b) where it does not vanish, and the vanishing condition zop
// (0 never, 1 a = 1, 2 a = 0, 3 b = 1, 4 b = 0).  za / zb: a / b is the zero
// parity; same: a and b are the same parity.
struct SlDec {
  bool ok = false, dead = false;
  int j00 = 0, da = 0, db = 0, dab = 0, zop = 0;
};

SlDec sliced_decompose(const Lut& l, bool za, bool zb, bool same) {
  SlDec r;
  if (l.spread != 0) return r;  // magnitude depends on the shot
  bool reach[2][2], zero[2][2];
  int jv[2][2];
  int nreach = 0, nzero = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      reach[a][b] = (!za || a == 0) && (!zb || b == 0) && (!same || a == b);
      const uint32_t inc = l.inc[a | (b << 1)];
      zero[a][b] = (inc >> 21) != 0;
      jv[a][b] = (int)(inc & 0x7FF) & 7;
      nreach += reach[a][b];
      nzero += reach[a][b] && zero[a][b];
    }
  r.ok = true;
  if (nzero == nreach) { r.dead = true; return r; }
  if (nzero) {
    auto fits = [&](int op) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          if (!reach[a][b]) continue;
          const bool want = op == 1 ? a == 1 : op == 2 ? a == 0 : op == 3 ? b == 1 : b == 0;
          if (zero[a][b] != want) return false;
        }
      return true;
    };
    r.zop = 0;
    for (int op = 1; op <= 4 && !r.zop; ++op) {
      if ((op <= 2 && za) || (op >= 3 && zb)) continue;
      if (fits(op)) r.zop = op;
    }
    if (!r.zop) { r.ok = false; return r; }
  }
  // fewest nonzero increments that reproduce J on the non-vanishing entries
  int best = 99;
  for (int dab = 0; dab <= 4; dab += 4)
    for (int da = 0; da < 8; ++da)
      for (int db = 0; db < 8; ++db)
        for (int j00 = 0; j00 < 8; ++j00) {
          if (za && (da || dab)) continue;           // a is always 0
          if (zb && (db || dab)) continue;           // b is always 0
          if (same && (db || dab)) continue;         // a = b: all of it in da
          bool ok = true;
          for (int a = 0; a < 2 && ok; ++a)
            for (int b = 0; b < 2 && ok; ++b)
              if (reach[a][b] && !zero[a][b]) ok = ((j00 + da * a + db * b + dab * a * b) & 7) == jv[a][b];
          const int cost = (da != 0) + (db != 0) + (dab != 0);
          if (ok && cost < best) {
            best = cost;
            r.j00 = j00;
            r.da = da;
            r.db = db;
            r.dab = dab;
          }
        }
  if (best == 99) r.ok = false;
  return r;
}

// Sliced form of one term (factor list f, coefficient phase j, magnitude
// exponent d); false when some factor has no such form.
template <class LutFn>
bool sliced_term(const std::vector<FacKey>& f, int j, int d, LutFn& lut, SlTerm& t) {
  // per host thread: programs compile in parallel threads without sharing it
  thread_local std::map<std::tuple<int, int, int, int>, SlDec> cache;
  t.d = d;
  int jc = j;
  std::map<uint32_t, int> delta;
  std::set<uint64_t> pairs;
  std::set<uint32_t> zp, zn;
  for (const FacKey& k : f) {
    const uint32_t qa = k.ia ? (uint32_t)k.ia + 1 : 0u, qb = k.ib ? (uint32_t)k.ib + 1 : 0u;
    const bool za = qa == 0, zb = qb == 0, same = qa != 0 && qa == qb;
    const int flags = (int)za | ((int)zb << 1) | ((int)same << 2);
    SlDec dec;
    {
      const auto key = std::make_tuple(k.kind, k.alpha & 7, k.beta & 7, flags);
      auto it = cache.find(key);
      if (it == cache.end()) it = cache.emplace(key, sliced_decompose(lut(k.kind, k.alpha, k.beta), za, zb, same)).first;
      dec = it->second;
    }
    if (!dec.ok) return false;
    if (dec.dead) { t.dead = true; return true; }
    jc += dec.j00;
    if (dec.da) delta[qa] = (delta[qa] + dec.da) & 7;
    if (dec.db) delta[qb] = (delta[qb] + dec.db) & 7;
    if (dec.dab) {
      const uint64_t key = (uint64_t)std::min(qa, qb) | ((uint64_t)std::max(qa, qb) << 32);
      if (!pairs.erase(key)) pairs.insert(key);  // (-1)^(ab) twice is 1
    }
    if (dec.zop == 1) zp.insert(qa);
    if (dec.zop == 2) zn.insert(qa);
    if (dec.zop == 3) zp.insert(qb);
    if (dec.zop == 4) zn.insert(qb);
  }
  for (uint32_t q : zp)
    if (zn.count(q)) { t.dead = true; return true; }
  t.j = jc & 7;
  // table-wide parity indices q (qa | qb << 32 for pi-pairs)
  for (const auto& [q, dl] : delta) {
    if (dl & 1) t.ops[SL_ADD1].push_back(q);
    const int rem = dl & 6;
    if (rem == 2) t.ops[SL_ADD2].push_back(q);
    if (rem == 4) t.ops[SL_XOR4].push_back(q);
    if (rem == 6) t.ops[SL_ADD6].push_back(q);
  }
  for (uint64_t pq : pairs) t.ops[SL_XOR4AB].push_back(pq);
  for (uint32_t q : zp) t.ops[SL_ZERO].push_back(q);
  for (uint32_t q : zn) t.ops[SL_ZEROC].push_back(q);
  return true;
}

// Local search after the greedy bank assignment of a segment's parity words.
// Each warp-wide parity load reads one word per lane; distinct words in one
// bank are served one after another, so a load costs the largest number of
// distinct words any bank holds for it.  Every load of the segment (a row's
// words, or for pi-pairs each half) is one group; a parity moves to a bank
// with a free slot when that lowers the summed cost of the groups it is in.
// A few passes; the moves never change which parity a row reads.
void refine_banks(const std::vector<std::array<uint64_t, 32>>& prow, const std::vector<int>& prow_code,
                  std::unordered_map<uint32_t, uint32_t>& slot, uint32_t fill[32], uint32_t cap) {
  // groups: distinct movable parities of one load
  std::vector<std::vector<uint32_t>> groups;
  groups.reserve(prow.size() * 2);
  for (size_t ri = 0; ri < prow.size(); ++ri) {
    for (int half = 0; half < (prow_code[ri] == SL_XOR4AB ? 2 : 1); ++half) {
      std::vector<uint32_t> g;
      for (uint64_t v : prow[ri]) {
        const uint32_t q = half ? (uint32_t)(v >> 32) : (uint32_t)v;
        if (q > kSlOnes) g.push_back(q);
      }
      std::sort(g.begin(), g.end());
      g.erase(std::unique(g.begin(), g.end()), g.end());
      if (g.size() > 1) groups.push_back(std::move(g));
    }
  }
  if (groups.empty()) return;
  std::unordered_map<uint32_t, std::vector<uint32_t>> member;  // parity -> its groups
  for (uint32_t gi = 0; gi < groups.size(); ++gi)
    for (uint32_t q : groups[gi]) member[q].push_back(gi);
  // per group: distinct words per bank, the largest count and how many banks reach it
  std::vector<std::array<uint8_t, 32>> cnt(groups.size());
  std::vector<uint8_t> mx(groups.size(), 0), nmx(groups.size(), 0);
  auto recount = [&](uint32_t gi) {
    uint8_t m = 0, n = 0;
    for (int b = 0; b < 32; ++b) {
      if (cnt[gi][(size_t)b] > m) {
        m = cnt[gi][(size_t)b];
        n = 1;
      } else if (cnt[gi][(size_t)b] == m) {
        ++n;
      }
    }
    mx[gi] = m;
    nmx[gi] = n;
  };
  for (uint32_t gi = 0; gi < groups.size(); ++gi) {
    cnt[gi].fill(0);
    for (uint32_t q : groups[gi]) cnt[gi][slot.at(q) & 31]++;
    recount(gi);
  }
  // free slots per bank (slot = bank + 32 x row, rows below cap)
  std::vector<std::vector<uint32_t>> freeslots(32);
  {
    std::vector<char> taken((size_t)32 * cap, 0);
    for (const auto& kv : slot)
      if (kv.second < 32u * cap) taken[kv.second] = 1;
    for (uint32_t sl = 2; sl < 32u * cap; ++sl)
      if (!taken[sl]) freeslots[sl & 31].push_back(sl);
  }
  std::vector<uint32_t> order;
  for (const auto& kv : member) order.push_back(kv.first);
  std::sort(order.begin(), order.end());
  for (int pass = 0; pass < 4; ++pass) {
    int moved = 0;
    for (uint32_t q : order) {
      const uint32_t a = slot.at(q) & 31;
      const std::vector<uint32_t>& gs = member.at(q);
      // cost change of leaving bank a, per group
      long base = 0;
      for (uint32_t gi : gs) base -= (cnt[gi][a] == mx[gi] && nmx[gi] == 1) ? 1 : 0;
      long best = 0;
      int bb = -1;
      for (int b = 0; b < 32; ++b) {
        if ((uint32_t)b == a || freeslots[(size_t)b].empty()) continue;
        long d = base;
        for (uint32_t gi : gs) {
          // after leaving a, the group's largest count is mx or mx - 1
          const int m0 = (cnt[gi][a] == mx[gi] && nmx[gi] == 1) ? mx[gi] - 1 : mx[gi];
          d += (cnt[gi][(size_t)b] + 1 > m0) ? 1 : 0;
        }
        if (d < best) {
          best = d;
          bb = b;
        }
      }
      if (bb < 0) continue;
      const uint32_t ns = freeslots[(size_t)bb].back();
      freeslots[(size_t)bb].pop_back();
      freeslots[a].push_back(slot.at(q));
      slot[q] = ns;
      for (uint32_t gi : gs) {
        cnt[gi][a]--;
        cnt[gi][(size_t)bb]++;
        recount(gi);
      }
      ++moved;
    }
    if (!moved) break;
  }
  // the fill of each bank: one past its highest taken row
  for (int b = 0; b < 32; ++b) fill[b] = 0;
  for (const auto& kv : slot) fill[kv.second & 31] = std::max(fill[kv.second & 31], kv.second / 32 + 1);
}

void pack(const Program& p, DeviceTables& out, int64_t sliced_min, int stage_rows, int seg_par) {
  std::map<std::tuple<int, int, int>, Lut> lut_cache;
  auto lut = [&](int kind, int alpha, int beta) -> const Lut& {
    auto key = std::make_tuple(kind, alpha & 7, beta & 7);
    auto it = lut_cache.find(key);
    if (it != lut_cache.end()) return it->second;
    Lut l{};
    if (!factor_lut(kind, alpha, beta, l.inc, &l.smin, &l.spread))
      throw PackError{TSIM_ERR_INTERNAL, "factor value is not a monomial of bounded spread"};
    return lut_cache.emplace(key, l).first->second;
  };
  const int W = padded_words_or_zero(p.W);
  if (!W) throw PackError{TSIM_ERR_ARG, "per-shot vector wider than 2048 bits is not supported"};
  if ((int)p.chain_norm.size() > kMaxChains) throw PackError{TSIM_ERR_ARG, "too many autoregressive chains for the kernel"};
  Packer s;
  DeviceLayout& L = out.layout;
  L = DeviceLayout();
  L.W = W;
  // channels
  L.o_ch = s.section();
  {
    uint32_t thr_off = 0, sig_off = 0;
    for (const ProgChannel& c : p.channels) {
      DChan d{};
      d.n_out = (uint32_t)c.sig.size();
      d.thr_off = thr_off;
      d.sig_off = sig_off;
      d.thr0 = c.thr.empty() ? 0xFFFFFFFFu : c.thr[0];
      thr_off += (uint32_t)c.thr.size();
      sig_off += (uint32_t)(c.sig.size() * (size_t)W);
      s.put(&d, sizeof d);
      for (size_t w = 0; !c.sig.empty() && w < c.sig[0].size(); ++w)
        if (c.sig[0][w]) throw PackError{TSIM_ERR_INTERNAL, "channel outcome 0 must not flip anything"};
    }
  }
  // geometric-gap groups: descriptors, member channel indices, and per
  // group T_k = floor(T_{k-1} Q / 2^32) for k = 1..n (T_0 = 2^32)
  L.o_grp = s.section();
  {
    uint32_t moff = 0;
    for (const NoiseGroup& g : p.groups) {
      uint64_t tn = 1ull << 32;
      for (size_t k = 0; k < g.member.size(); ++k) tn = (tn * (uint64_t)g.Q) >> 32;
      DGroup d{g.Q, (uint32_t)g.member.size(), moff, (uint32_t)tn,
               (float)(1.0 / std::log2((double)g.Q / 4294967296.0))};
      moff += (uint32_t)g.member.size();
      s.put(&d, sizeof d);
    }
  }
  L.o_gmem = s.section();
  for (const NoiseGroup& g : p.groups)
    for (int c : g.member) {
      const uint32_t v = (uint32_t)c;
      s.put(&v, 4);
    }
  L.o_gT = s.section();
  for (const NoiseGroup& g : p.groups) {
    uint64_t t = 1ull << 32;
    for (size_t k = 0; k < g.member.size(); ++k) {
      t = (t * (uint64_t)g.Q) >> 32;
      const uint32_t v = (uint32_t)t;
      s.put(&v, 4);
    }
  }
  L.o_t0 = s.section();
  for (size_t i = 0; i < (p.channels.size() + 3) / 4 * 4; ++i) {
    const uint32_t t = i < p.channels.size() && !p.channels[i].thr.empty() ? p.channels[i].thr[0] : 0xFFFFFFFFu;
    s.put(&t, 4);
  }
  L.o_thr = s.section();
  for (const ProgChannel& c : p.channels)
    for (uint32_t t : c.thr) s.put(&t, 4);
  { uint32_t z = 0; s.put(&z, 4); }
  L.o_sig = s.section();
  for (const ProgChannel& c : p.channels)
    for (const auto& sg : c.sig) s.put_padded(sg, W);
  // outputs; in detector mode consecutive single-bit outputs without a
  // constant on consecutive X bits, in the same record, become one run
  L.o_out = s.section();
  {
    int32_t mo = 0;
    std::vector<DOut> ents;
    for (size_t i = 0; i < p.outputs.size(); ++i) {
      const ProgOutput& o = p.outputs[i];
      DOut d{};
      d.cst = o.cst;
      d.rec = (int32_t)i;
      if (o.random) {
        d.kind = OUT_RANDOM;
        d.a = o.xbit;
        d.chain = o.chain;
        d.table = o.table;
      } else {
        int ones = 0, pos = -1;
        for (size_t w = 0; w < o.mask.size(); ++w)
          for (int bb = 0; bb < 64; ++bb)
            if ((o.mask[w] >> bb) & 1) { ++ones; pos = (int)(w * 64 + (size_t)bb); }
        if (ones == 1) { d.kind = OUT_BIT; d.a = pos; }
        else { d.kind = OUT_MASK; d.a = mo; }
      }
      mo += W;
      if (p.mode == TSIM_MODE_DETECTORS && d.kind == OUT_BIT && d.cst == 0 && !ents.empty()) {
        DOut& prev = ents.back();
        const bool same_rec = ((int)i < p.ndet) == (prev.rec < p.ndet);
        if (same_rec && prev.kind == OUT_BIT && prev.cst == 0 && prev.a + 1 == d.a && prev.rec + 1 == d.rec) {
          prev.kind = OUT_RUN;
          prev.chain = 2;
          continue;
        }
        if (same_rec && prev.kind == OUT_RUN && prev.a + prev.chain == d.a && prev.rec + prev.chain == d.rec) {
          prev.chain++;
          continue;
        }
      }
      ents.push_back(d);
    }
    if (!ents.empty()) s.put(ents.data(), ents.size() * sizeof(DOut));
    L.n_ent = (int)ents.size();
    for (const DOut& d : ents)
      if (d.kind == OUT_RUN) {
        L.runs++;
        L.run_outputs += (uint64_t)d.chain;
      }
  }
  L.o_om = s.section();
  for (const ProgOutput& o : p.outputs) s.put_padded(o.mask, W);
  L.o_cn = s.section();
  for (int c : p.chain_norm) { int32_t v = c; s.put(&v, 4); }
  { int32_t z = 0; s.put(&z, 4); }
  // a chain with a table of arbitrary phases is evaluated in floating point,
  // all its tables with it (Algorithm 1 needs one arithmetic per chain)
  std::vector<char> chain_fl(p.chain_norm.size(), 0), tab_fl(p.tables.size(), 0);
  for (size_t c = 0; c < p.chain_norm.size(); ++c) chain_fl[c] = p.tables[(size_t)p.chain_norm[c]].is_float();
  for (const ProgOutput& o : p.outputs)
    if (o.random && p.tables[(size_t)o.table].is_float()) chain_fl[(size_t)o.chain] = 1;
  for (size_t c = 0; c < p.chain_norm.size(); ++c)
    if (chain_fl[c]) tab_fl[(size_t)p.chain_norm[c]] = 1;
  for (const ProgOutput& o : p.outputs)
    if (o.random && chain_fl[(size_t)o.chain]) tab_fl[(size_t)o.table] = 1;
  L.o_cf = s.section();
  for (char f : chain_fl) { int32_t v = f; s.put(&v, 4); }
  { int32_t z = 0; s.put(&z, 4); }

  // tables: distinct parities, then terms merged into classes with equal factors
  struct Cls {
    std::vector<FacKey> f;
    ZW coef;
  };
  std::vector<DTable> tabs;
  std::vector<uint64_t> par;
  std::vector<DClass> cls;
  std::vector<uint32_t> fidx, finc;
  std::vector<uint64_t> fcoord;
  std::vector<DSBatch> sbs;
  std::vector<DSeg> segs;
  std::vector<uint32_t> rows;
  std::vector<uint32_t> ffidx;
  std::vector<double> ffang;
  for (size_t ti = 0; ti < p.tables.size(); ++ti) {
    const ProgTable& tb = p.tables[ti];
    DTable dt{};
    dt.par_off = (uint32_t)(par.size() / (size_t)W);
    std::map<std::vector<uint64_t>, int> pidx;
    std::vector<std::vector<uint64_t>> plist;
    auto parity_index = [&](const std::vector<uint64_t>& m) {
      std::vector<uint64_t> key((size_t)W, 0);
      for (size_t i = 0; i < m.size() && i < (size_t)W; ++i) key[i] = m[i];
      auto it = pidx.find(key);
      if (it != pidx.end()) return it->second;
      int id = (int)plist.size();
      pidx[key] = id;
      plist.push_back(key);
      return id;
    };
    parity_index(std::vector<uint64_t>((size_t)W, 0));  // index 0: the zero parity
    if (tab_fl[ti]) {
      // FLOAT: terms with equal factor lists merged, the complex coefficient
      // summed in double; exact factors as per-thread increments, arbitrary
      // ones as (parity, angle)
      std::map<std::vector<FacKey>, size_t> fidx_of;
      std::vector<std::pair<std::vector<FacKey>, std::complex<double>>> fcl;
      for (const ProgTerm& tm : tb.terms) {
        std::vector<FacKey> fk;
        for (const ProgFactor& f : tm.f) {
          FacKey k{f.kind, f.kind == 4 ? 0 : (f.alpha & 7), f.kind == 4 ? 0 : (f.beta & 7), parity_index(f.u),
                   f.kind == 4 ? 0 : parity_index(f.v)};
          k.t = f.kind == 4 ? f.t : 0.0;
          fk.push_back(k);
        }
        std::sort(fk.begin(), fk.end());
        ZW c0 = ZW::omega(tm.j0);
        c0.k = tm.s0;
        const std::complex<double> c = zw_to_complex(c0) * std::polar(1.0, M_PI * tm.fph);
        auto it = fidx_of.find(fk);
        if (it == fidx_of.end()) {
          fidx_of[fk] = fcl.size();
          fcl.push_back({fk, c});
        } else {
          fcl[it->second].second += c;
        }
      }
      if (plist.size() > (size_t)kMaxParities)
        throw PackError{TSIM_ERR_ARG, "a floating-point table has more than 256 distinct parities"};
      dt.mode = TAB_FLOAT;
      dt.base = 0;
      dt.par_off = (uint32_t)(par.size() / (size_t)W);
      for (const auto& m : plist) par.insert(par.end(), m.begin(), m.end());
      dt.n_par = (uint32_t)plist.size();
      dt.cls_off = (uint32_t)cls.size();
      uint64_t nfac = 0;
      for (const auto& [fk, coef] : fcl) {
        DClass d{};
        d.fac_off = (uint32_t)fidx.size();
        d.mono = 2;
        d.j0 = (int32_t)ffidx.size();
        int smin_sum = 0;
        for (const FacKey& k : fk) {
          if (k.kind == 4) {
            ffidx.push_back((uint32_t)k.ia);
            ffang.push_back(k.t);
            continue;
          }
          const Lut& l = lut(k.kind, k.alpha, k.beta);
          smin_sum += l.smin;
          fidx.push_back((uint32_t)k.ia | ((uint32_t)k.ib << 8));
          finc.insert(finc.end(), l.inc, l.inc + 4);
          fcoord.push_back(0);
          fcoord.push_back(0);
          d.n_fac++;
        }
        d.pad = (int32_t)(ffidx.size() - (size_t)d.j0);
        const std::complex<double> cc = coef * std::pow(std::sqrt(2.0), smin_sum);
        double re = cc.real(), im = cc.imag();
        std::memcpy(&d.c[0], &re, 8);
        std::memcpy(&d.c[1], &im, 8);
        nfac += fk.size();
        cls.push_back(d);
      }
      dt.n_cls = (uint32_t)fcl.size();
      L.classes += fcl.size();
      L.parities += plist.size() - 1;
      L.table_classes.push_back(fcl.size());
      L.table_parities.push_back(plist.size() - 1);
      L.table_class_factors.push_back(nfac);
      L.class_factors += nfac;
      L.table_mode.push_back(TAB_FLOAT);
      L.table_batches.push_back(0);
      L.table_rows.push_back(0);
      L.table_ops.push_back(0);
      L.table_work32.push_back(0);
      L.table_work32_real.push_back(0);
      tabs.push_back(dt);
      continue;
    }
    std::map<std::vector<FacKey>, size_t> cidx;
    std::vector<Cls> cl;
    for (const ProgTerm& tm : tb.terms) {
      std::vector<FacKey> fk;
      for (const ProgFactor& f : tm.f) {
        FacKey k{f.kind, f.alpha & 7, f.beta & 7, parity_index(f.u), parity_index(f.v)};
        fk.push_back(k);
      }
      std::sort(fk.begin(), fk.end());
      ZW c = ZW::omega(tm.j0);
      c.k = tm.s0;
      auto it = cidx.find(fk);
      if (it == cidx.end()) {
        cidx[fk] = cl.size();
        cl.push_back({fk, c});
      } else {
        cl[it->second].coef = zw_add(cl[it->second].coef, c);
      }
    }
    // per class: exponent of its smallest possible magnitude
    struct Prep { size_t i; int raw, spread, mono, j, zero; };
    std::vector<Prep> prep;
    for (size_t i = 0; i < cl.size(); ++i) {
      if (cl[i].coef.zero()) continue;  // exact cancellation between terms
      if (cl[i].f.size() > 255) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "term with more than 255 factors"};
      int smin_sum = 0, spread = 0;
      for (const FacKey& k : cl[i].f) {
        const Lut& l = lut(k.kind, k.alpha, k.beta);
        smin_sum += l.smin;
        spread += l.spread;
      }
      int z, ms, mj;
      Prep pr{i, 0, spread, 0, 0, 0};
      if (monomial_of(cl[i].coef, &z, &ms, &mj)) {
        pr.mono = 1;
        pr.j = mj;
        pr.raw = ms + smin_sum;
      } else {
        pr.raw = cl[i].coef.k + smin_sum;
      }
      prep.push_back(pr);
    }
    int base = 0;
    for (size_t q = 0; q < prep.size(); ++q) base = q ? std::min(base, prep[q].raw) : prep[q].raw;
    dt.base = base;
    dt.n_cls = (uint32_t)prep.size();
    // every coefficient of the accumulated sum stays below 2^62 in absolute value
    unsigned __int128 bound = 0;
    for (const Prep& pr : prep) {
      const Cls& c = cl[pr.i];
      unsigned __int128 mag = 1;
      if (!pr.mono) {
        mag = 0;
        for (int i = 0; i < 4; ++i) {
          if (c.coef.c[i] > ((__int128)1 << 60) || c.coef.c[i] < -((__int128)1 << 60))
            throw PackError{TSIM_ERR_OVERFLOW_BOUND, "merged term coefficient exceeds 60 bits"};
          mag += (unsigned __int128)(c.coef.c[i] < 0 ? -c.coef.c[i] : c.coef.c[i]);
        }
        mag *= 2;  // the sqrt2 multiplication at most doubles the largest coefficient
      }
      const int dm = pr.raw - base + pr.spread;
      if (dm / 2 + log2_ceil(mag) >= 100) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "table magnitudes exceed 64-bit accumulation"};
      bound += mag << (dm / 2 + 1);
    }
    if (bound >= ((unsigned __int128)1 << 62)) throw PackError{TSIM_ERR_OVERFLOW_BOUND, "table magnitudes exceed 64-bit accumulation"};

    // ---- bit-sliced layout (large tables whose factors all reduce to
    // operations on J and Z, every term a monomial)
    bool sliced = sliced_min >= 0 && prep.size() >= (size_t)std::max<int64_t>(sliced_min, 1);
    std::vector<SlTerm> sterms;
    for (size_t q = 0; sliced && q < prep.size(); ++q) {
      const Prep& pr = prep[q];
      if (!pr.mono) { sliced = false; break; }
      SlTerm t;
      if (!sliced_term(cl[pr.i].f, pr.j, pr.raw - base, lut, t)) { sliced = false; break; }
      if (!t.dead) sterms.push_back(std::move(t));
    }
    uint64_t real_ops = 0, padded_rows = 0, sliced_work = 0, nbatches = 0, real_work = 0;
    if (sliced) {
      dt.mode = TAB_SLICED;
      dt.sb_off = (int32_t)segs.size();  // sliced: the table's segments
      // integer lane-operations of one warp (32 shots) on this table: the
      // bit transpose of X (W paired transposes of 5 stages of 6 ops, and 2W
      // stores, 32 lanes), per segment each parity (load, store, and per mask
      // bit: find, load, XOR), each padded row on 32 lanes (its share of the
      // 16-byte row load and of the code dispatch, its parity load(s) and the
      // word operations of its code), and per batch 2 paired transposes, the
      // signed counts and their accumulation (about 90 per lane).
      // real_work counts the same operations without padding: the rows of
      // each term's own factors and one batch epilogue per term (lane).
      static const int kRowOps[kSlCodes] = {3, 4, 5, 4, 3, 3, 6};
      constexpr uint64_t kBatchOps = 90;
      uint64_t w32 = 32ull * 32 * (uint64_t)W;
      uint64_t wreal = w32;
      uint32_t most = 0;
      auto parities_of = [](const SlTerm& t, std::vector<uint32_t>& out) {
        out.clear();
        for (int c = 0; c < kSlCodes; ++c)
          for (uint64_t r : t.ops[c]) {
            out.push_back((uint32_t)r);
            if (c == SL_XOR4AB) out.push_back((uint32_t)(r >> 32));
          }
      };
      // segments: consecutive terms (the decomposition's order keeps their
      // parities local) while the parity list stays within seg_par words
      std::vector<uint32_t> tp;
      for (size_t t0 = 0; t0 < sterms.size();) {
        std::set<uint32_t> ps;
        size_t t1 = t0;
        while (t1 < sterms.size()) {
          parities_of(sterms[t1], tp);
          size_t add = 0;
          for (uint32_t q : tp) add += q > kSlOnes && !ps.count(q);
          if (t1 > t0 && ps.size() + add + 2 > (size_t)seg_par) break;
          for (uint32_t q : tp)
            if (q > kSlOnes) ps.insert(q);
          ++t1;
        }
        if (ps.size() + 2 > (size_t)kSlMaxPar) throw PackError{TSIM_ERR_ARG, "a sliced term has too many parities"};
        // the segment's terms, sorted by magnitude then by operation counts
        // (so that a batch's terms need similar numbers of rows per code)
        std::vector<SlTerm> lt(sterms.begin() + (long)t0, sterms.begin() + (long)t1);
        std::stable_sort(lt.begin(), lt.end(), [](const SlTerm& a, const SlTerm& b) {
          if (a.d != b.d) return a.d < b.d;
          size_t na = 0, nb = 0;
          for (int c = 0; c < kSlCodes; ++c) { na += a.ops[c].size(); nb += b.ops[c].size(); }
          if (na != nb) return na > nb;
          for (int c = 0; c < kSlCodes; ++c)
            if (a.ops[c].size() != b.ops[c].size()) return a.ops[c].size() > b.ops[c].size();
          return false;
        });
        // batches of 32 terms and their rows, as table-wide parity indices
        // (0 and kSlOnes for padding, qa | qb << 32 for pi-pairs)
        struct PBatch {
          size_t b0, b1;
          uint16_t cnt[kSlCodes];
        };
        std::vector<PBatch> pb;
        std::vector<std::array<uint64_t, 32>> prow;
        std::vector<int> prow_code;
        for (size_t b0 = 0; b0 < lt.size();) {
          size_t b1 = b0;
          while (b1 < lt.size() && b1 - b0 < 32 && lt[b1].d == lt[b0].d) ++b1;
          PBatch B{b0, b1, {}};
          for (int c = 0; c < kSlCodes; ++c) {
            size_t n = 0;
            for (size_t l = b0; l < b1; ++l) n = std::max(n, lt[l].ops[c].size());
            n = (n + 3) & ~(size_t)3;  // whole groups of 4 rows: no single-row tail loop on the device
            if (n > 0xFFFF) throw PackError{TSIM_ERR_ARG, "too many operations of one kind in a term"};
            B.cnt[c] = (uint16_t)n;
            for (size_t k = 0; k < n; ++k) {
              std::array<uint64_t, 32> r;
              for (size_t l = 0; l < 32; ++l) {
                const size_t ti = b0 + l;
                r[l] = (ti < b1 && k < lt[ti].ops[c].size()) ? lt[ti].ops[c][k] : (c == SL_ZEROC ? kSlOnes : 0u);
              }
              prow.push_back(r);
              prow_code.push_back(c);
            }
          }
          pb.push_back(B);
          b0 = b1;
        }
        // shared-memory slot of every parity: word q of the buffer lies in
        // bank q mod 32, and the 32 lanes of a row read their words at once,
        // so distinct parities of one row go to distinct banks where possible
        // (greedy, in row order; slot = bank + 32 x fill)
        std::unordered_map<uint32_t, uint32_t> slot;
        slot.reserve(ps.size() * 2 + 4);
        slot[0] = 0;
        slot[kSlOnes] = kSlOnes;
        uint32_t fill[32] = {0};
        fill[0] = fill[1] = 1;
        const uint32_t cap = (uint32_t)((ps.size() + 2 + 31) / 32) + 1;
        for (size_t ri = 0; ri < prow.size(); ++ri) {
          uint32_t qs[64];
          int nq = 0;
          for (uint64_t v : prow[ri]) {
            qs[nq++] = (uint32_t)v;
            if (prow_code[ri] == SL_XOR4AB && (v >> 32)) qs[nq++] = (uint32_t)(v >> 32);
          }
          std::sort(qs, qs + nq);
          nq = (int)(std::unique(qs, qs + nq) - qs);
          int used[32] = {0};
          for (int k = 0; k < nq; ++k) {
            auto it = slot.find(qs[k]);
            if (it != slot.end()) used[it->second & 31]++;
          }
          for (int k = 0; k < nq; ++k) {
            if (slot.count(qs[k])) continue;
            int best = -1;
            for (int b = 0; b < 32; ++b)
              if (fill[b] < cap && (best < 0 || used[b] < used[best] || (used[b] == used[best] && fill[b] < fill[best])))
                best = b;
            slot[qs[k]] = (uint32_t)best + 32u * fill[best];
            fill[best]++;
            used[best]++;
          }
        }
        refine_banks(prow, prow_code, slot, fill, cap);
        uint32_t nslot = 2;
        for (const auto& kv : slot) nslot = std::max(nslot, kv.second + 1);
        if (nslot > (uint32_t)kSlMaxPar) throw PackError{TSIM_ERR_ARG, "a sliced term has too many parities"};
        DSeg g{};
        g.par_off = (uint32_t)(par.size() / (size_t)W);
        g.n_par = nslot;
        {
          std::vector<uint32_t> of_slot(nslot, 0);  // table parity index per slot (0: none)
          for (const auto& kv : slot)
            if (kv.first > kSlOnes) of_slot[kv.second] = kv.first;
          for (uint32_t sl = 0; sl < nslot; ++sl) {
            // slot 0: the zero parity; kSlOnes: all ones (set on the device);
            // unused slots: zero masks
            if (of_slot[sl]) par.insert(par.end(), plist[of_slot[sl] - 1].begin(), plist[of_slot[sl] - 1].end());
            else par.insert(par.end(), (size_t)W, 0ull);
          }
        }
        for (uint32_t q : ps) {
          uint64_t pop = 0;
          for (uint64_t m : plist[q - 1]) pop += (uint64_t)__builtin_popcountll(m);
          w32 += 3 + 3 * pop;
          wreal += 3 + 3 * pop;
        }
        w32 += 3 * (uint64_t)(nslot - ps.size());
        // rows hold byte offsets of the slots' words: 4 slot, or
        // 4 slot_a | 4 slot_b << 16 for pi-pairs; groups of 4 rows are
        // [group][lane][4], so a lane's 4 rows are 16 contiguous bytes
        g.sb_off = (uint32_t)sbs.size();
        size_t ri = 0;
        for (const PBatch& P : pb) {
          DSBatch B{};
          B.row_off = (uint32_t)rows.size();
          B.d = lt[P.b0].d;
          for (size_t l = 0; l < P.b1 - P.b0; ++l) {
            const SlTerm& t = lt[P.b0 + l];
            B.valid |= 1u << l;
            for (int bit = 0; bit < 3; ++bit) B.j0m[bit] |= (uint32_t)((t.j >> bit) & 1) << l;
          }
          uint32_t nrows = 0;
          for (int c = 0; c < kSlCodes; ++c) {
            const size_t n = P.cnt[c];
            B.cnt[c] = (uint16_t)n;
            for (size_t gi = 0; gi < n / 4; ++gi)
              for (size_t l = 0; l < 32; ++l)
                for (size_t k = 4 * gi; k < 4 * gi + 4; ++k) {
                  const uint64_t v = prow[ri + k][l];
                  uint32_t r;
                  if (c == SL_XOR4AB) r = (4 * slot.at((uint32_t)v)) | ((4 * slot.at((uint32_t)(v >> 32))) << 16);
                  else r = 4 * slot.at((uint32_t)v);
                  const size_t ti = P.b0 + l;
                  if (ti < P.b1 && k < lt[ti].ops[c].size()) {
                    ++real_ops;
                    wreal += (uint64_t)kRowOps[c];
                  }
                  rows.push_back(r);
                }
            ri += n;
            padded_rows += n;
            nrows += (uint32_t)n;
            w32 += (uint64_t)n * 32 * (uint64_t)kRowOps[c];
          }
          w32 += 32 * kBatchOps;
          wreal += kBatchOps * (uint64_t)(P.b1 - P.b0);
          most = std::max(most, nrows);
          if (rows.size() > 0xFFFFFFFFull) throw PackError{TSIM_ERR_ARG, "sliced tables too large"};
          sbs.push_back(B);
        }
        g.n_sb = (uint32_t)(sbs.size() - g.sb_off);
        nbatches += g.n_sb;
        L.sl_par_max = std::max<uint32_t>(L.sl_par_max, g.n_par);
        segs.push_back(g);
        t0 = t1;
      }
      dt.n_sb = (int32_t)(segs.size() - (size_t)dt.sb_off);
      dt.n_par = 0;
      // stage the rows through shared memory when every batch fits a buffer
      dt.stage = stage_rows > 0 && most <= (uint32_t)stage_rows ? 1 : 0;
      if (dt.stage) L.sl_rows_max = std::max(L.sl_rows_max, most);
      sliced_work = w32;
      real_work = wreal;
    } else {
      // few distinct parities: evaluate each once per shot and index them;
      // many: evaluate a GF(2) basis of their span and give every parity its
      // coordinates in that basis
      std::vector<uint64_t> coords(plist.size(), 0);
      dt.par_off = (uint32_t)(par.size() / (size_t)W);
      if (plist.size() <= (size_t)kMaxParities) {
        for (const auto& m : plist) par.insert(par.end(), m.begin(), m.end());
        dt.n_par = (uint32_t)plist.size();
      } else {
        dt.mode = TAB_BASIS;
        std::vector<std::vector<uint64_t>> bvec, borig;
        std::vector<uint64_t> bcomb;
        std::vector<int> bpiv;
        for (size_t i = 1; i < plist.size(); ++i) {
          std::vector<uint64_t> v = plist[i];
          uint64_t comb = 0;
          for (size_t j = 0; j < bvec.size(); ++j)
            if ((v[(size_t)bpiv[j] >> 6] >> (bpiv[j] & 63)) & 1) {
              for (int w = 0; w < W; ++w) v[(size_t)w] ^= bvec[j][(size_t)w];
              comb ^= bcomb[j];
            }
          int piv = -1;
          for (int w = 0; w < W && piv < 0; ++w)
            if (v[(size_t)w]) piv = w * 64 + __builtin_ctzll(v[(size_t)w]);
          if (piv < 0) { coords[i] = comb; continue; }
          if (borig.size() >= 64) throw PackError{TSIM_ERR_ARG, "table parities span more than 64 dimensions"};
          const uint64_t me = 1ull << borig.size();
          borig.push_back(plist[i]);
          bvec.push_back(v);
          bcomb.push_back(comb ^ me);
          bpiv.push_back(piv);
          coords[i] = me;
        }
        for (const auto& m : borig) par.insert(par.end(), m.begin(), m.end());
        dt.n_par = (uint32_t)borig.size();
      }
      const bool basis = dt.mode == TAB_BASIS;
      dt.cls_off = (uint32_t)cls.size();
      for (const Prep& pr : prep) {
        const Cls& c = cl[pr.i];
        DClass d{};
        d.fac_off = (uint32_t)fidx.size();
        d.n_fac = (uint32_t)c.f.size();
        d.mono = pr.mono;
        d.j0 = pr.j;
        d.d0 = pr.raw - base;
        if (!pr.mono)
          for (int i = 0; i < 4; ++i) d.c[i] = (long long)c.coef.c[i];
        for (const FacKey& k : c.f) {
          const Lut& l = lut(k.kind, k.alpha, k.beta);
          fidx.push_back(basis ? 0u : ((uint32_t)k.ia | ((uint32_t)k.ib << 8)));
          finc.insert(finc.end(), l.inc, l.inc + 4);
          fcoord.push_back(basis ? coords[(size_t)k.ia] : 0);
          fcoord.push_back(basis ? coords[(size_t)k.ib] : 0);
        }
        cls.push_back(d);
      }
    }
    L.classes += prep.size();
    L.parities += plist.size() - 1;
    L.table_classes.push_back(prep.size());
    L.table_parities.push_back(plist.size() - 1);
    {
      uint64_t nf = 0;
      for (const Prep& pr : prep) nf += cl[pr.i].f.size();
      L.table_class_factors.push_back(nf);
      L.class_factors += nf;
    }
    L.table_mode.push_back(dt.mode);
    L.table_batches.push_back(nbatches);
    L.table_rows.push_back(padded_rows);
    L.table_ops.push_back(real_ops);
    L.table_work32.push_back(sliced_work);
    L.table_work32_real.push_back(real_work);
    tabs.push_back(dt);
  }
  // tables whose value does not depend on the shot (only the zero parity):
  // the value at the table base, and for a chain normalisation the power of
  // w that makes it real and positive
  std::vector<DConst> tconst(tabs.size(), DConst{});
  {
    std::vector<char> is_norm(tabs.size(), 0);
    for (int c : p.chain_norm) is_norm[(size_t)c] = 1;
    const std::vector<uint64_t> zeros((size_t)W, 0);
    for (size_t t = 0; t < tabs.size(); ++t) {
      DTable& dt = tabs[t];
      dt.cst = 0;
      dt.rot = -1;
      if (dt.mode != TAB_SCALAR || dt.n_par != 1) continue;
      ZW v = eval_table_host(p, (int)t, zeros.data());
      if (v.zero()) v.k = dt.base;
      if (v.k < dt.base) continue;
      while (v.k > dt.base) v = zw_lower_k(v);
      bool fits = true;
      for (int i = 0; i < 4; ++i) fits = fits && v.c[i] < ((__int128)1 << 62) && v.c[i] > -((__int128)1 << 62);
      if (!fits) continue;
      for (int i = 0; i < 4; ++i) tconst[t].c[i] = (long long)v.c[i];
      dt.cst = 1;
      if (!is_norm[t]) continue;
      for (int rot = 0; rot < 8 && dt.rot < 0; ++rot) {
        ZW r = zw_mul(v, ZW::omega(-rot));
        if (r.c[2] != 0 || r.c[1] + r.c[3] != 0) continue;
        // Re = (2 c0 + (c1 - c3) sqrt2) / 2 > 0
        const __int128 X = 2 * r.c[0], Y = r.c[1] - r.c[3];
        bool pos;
        if (X >= 0 && Y >= 0) pos = X > 0 || Y > 0;
        else if (X <= 0 && Y <= 0) pos = false;
        else {
          // compare X^2 with 2 Y^2 exactly (both below 2^126 under the bound)
          const unsigned __int128 ax = (unsigned __int128)(X < 0 ? -X : X), ay = (unsigned __int128)(Y < 0 ? -Y : Y);
          if ((ax >> 62) || (ay >> 62)) continue;  // left to the device
          const unsigned __int128 x2 = ax * ax, y2 = 2 * ay * ay;
          pos = X > 0 ? x2 > y2 : y2 > x2;
        }
        if (pos) dt.rot = rot;
      }
    }
  }
  L.o_tc = s.section();
  if (!tconst.empty()) s.put(tconst.data(), tconst.size() * sizeof(DConst));
  L.o_tab = s.section();
  if (!tabs.empty()) s.put(tabs.data(), tabs.size() * sizeof(DTable));
  L.o_par = s.section();
  if (!par.empty()) s.put(par.data(), par.size() * 8);
  // per parity slot, its X bits as eight 8-bit indices when it has at most
  // eight (X of at most 4 words; unused entries name an X bit that is always
  // 0, past the program's n_x), else .x = kSlWalk: the kernel then walks the
  // slot's mask.  Bit-sliced segments form their parity words from these
  // with four (k8 = 0) or eight shared loads instead of a loop over the mask.
  {
    std::vector<uint2> pidx(par.size() / (size_t)W, make_uint2(kSlWalk, kSlWalk));
    std::vector<uint8_t> wide(pidx.size(), 0);
    const int zb = p.nx < 64 * W ? 64 * W - 1 : -1;
    if (W <= 4 && zb >= 0)
      for (size_t q = 0; q < pidx.size(); ++q) {
        int bits[8], nb = 0;
        bool ok = true;
        for (int w = 0; w < W && ok; ++w)
          for (uint64_t m = par[q * (size_t)W + (size_t)w]; m && ok; m &= m - 1) {
            if (nb == 8) ok = false;
            else bits[nb++] = 64 * w + __builtin_ctzll(m);
          }
        if (!ok) continue;
        uint32_t v[2] = {0, 0};
        for (int k = 0; k < 8; ++k) v[k >> 2] |= (uint32_t)(k < nb ? bits[k] : zb) << (8 * (k & 3));
        if (v[0] == kSlWalk) continue;  // only when zb is 255 and no bit is named: walk the (zero) mask
        pidx[q] = make_uint2(v[0], v[1]);
        wide[q] = nb > 4;
      }
    for (DSeg& g : segs) {
      g.k8 = 0;
      for (uint32_t q = 0; q < g.n_par; ++q) g.k8 |= wide[(size_t)g.par_off + q];
    }
    L.o_pidx = s.section();
    if (!pidx.empty()) s.put(pidx.data(), pidx.size() * sizeof(uint2));
  }
  L.o_cls = s.section();
  if (!cls.empty()) s.put(cls.data(), cls.size() * sizeof(DClass));
  L.o_fidx = s.section();
  if (!fidx.empty()) s.put(fidx.data(), fidx.size() * 4);
  L.o_finc = s.section();
  if (!finc.empty()) s.put(finc.data(), finc.size() * 4);
  L.o_fco = s.section();
  if (!fcoord.empty()) s.put(fcoord.data(), fcoord.size() * 8);
  L.o_seg = s.section();
  if (!segs.empty()) s.put(segs.data(), segs.size() * sizeof(DSeg));
  L.o_sb = s.section();
  if (!sbs.empty()) s.put(sbs.data(), sbs.size() * sizeof(DSBatch));
  L.o_row = s.section();
  if (!rows.empty()) s.put(rows.data(), rows.size() * 4);
  L.o_ffi = s.section();
  if (!ffidx.empty()) s.put(ffidx.data(), ffidx.size() * 4);
  L.o_ffa = s.section();
  if (!ffang.empty()) s.put(ffang.data(), ffang.size() * 8);
  L.sl_par = L.sl_par_max ? (int)((L.sl_par_max + 3) & ~3u) : 0;
  L.sl_rb = (int)L.sl_rows_max * 32;
  // measurement-mode detector / observable maps (CSR)
  auto csr = [&](const std::vector<std::vector<int>>& m, size_t* o_off, size_t* o_idx) {
    *o_off = s.section();
    int32_t acc = 0;
    s.put(&acc, 4);
    for (const auto& d : m) { acc += (int32_t)d.size(); s.put(&acc, 4); }
    *o_idx = s.section();
    for (const auto& d : m)
      for (int j : d) { int32_t v = j; s.put(&v, 4); }
    int32_t z = 0;
    s.put(&z, 4);
  };
  csr(p.detmap, &L.o_dmo, &L.o_dmi);
  csr(p.obsmap, &L.o_omo, &L.o_omi);
  // measurement mode: every detector / observable (Eq. xor) as one parity of
  // X: the XOR of its measurements' vectors (a deterministic output's mask, a
  // random output's own X bit) and of their constants; X keeps every drawn
  // bit until the shot ends, so the parity at the end equals the XOR
  auto xor_masks = [&](const std::vector<std::vector<int>>& m, size_t* o_mask, size_t* o_cst) {
    std::vector<uint64_t> masks;
    std::vector<int32_t> csts;
    for (const auto& d : m) {
      std::vector<uint64_t> mk((size_t)W, 0);
      int c = 0;
      for (int j : d) {
        const ProgOutput& o = p.outputs[(size_t)j];
        if (o.random) {
          mk[(size_t)o.xbit >> 6] ^= 1ull << (o.xbit & 63);
        } else {
          for (size_t w = 0; w < o.mask.size() && w < (size_t)W; ++w) mk[w] ^= o.mask[w];
          c ^= o.cst;
        }
      }
      masks.insert(masks.end(), mk.begin(), mk.end());
      csts.push_back(c);
    }
    *o_mask = s.section();
    if (!masks.empty()) s.put(masks.data(), masks.size() * 8);
    *o_cst = s.section();
    if (!csts.empty()) s.put(csts.data(), csts.size() * 4);
    int32_t z = 0;
    s.put(&z, 4);
  };
  if (p.mode == TSIM_MODE_MEASUREMENTS) {
    xor_masks(p.detmap, &L.o_dmk, &L.o_dcs);
    xor_masks(p.obsmap, &L.o_omk, &L.o_ocs);
  }
  L.total = s.section();
  out.blob.swap(s.b);
}

DevView make_view(const unsigned char* base, const DeviceLayout& L, const Program& p) {
  DevView v{};
  v.W = L.W;
  v.n_ch = (int)p.channels.size();
  v.n_out = (int)p.outputs.size();
  v.n_ent = L.n_ent;
  v.n_chains = (int)p.chain_norm.size();
  v.n_tab = (int)p.tables.size();
  v.nmeas = p.nmeas;
  v.ndet = p.ndet;
  v.nobs = p.nobs;
  v.mode = p.mode;
  v.status = nullptr;  // set by the caller: the status word of the device the view lives on
  v.noise_mode = p.noise_mode;
  v.n_grp = (int)p.groups.size();
  v.grp = (const DGroup*)(base + L.o_grp);
  v.gmem = (const uint32_t*)(base + L.o_gmem);
  v.gT = (const uint32_t*)(base + L.o_gT);
  v.ch = (const DChan*)(base + L.o_ch);
  v.thr0 = (const uint4*)(base + L.o_t0);
  v.thr = (const uint32_t*)(base + L.o_thr);
  v.sig = (const uint64_t*)(base + L.o_sig);
  v.out = (const DOut*)(base + L.o_out);
  v.omask = (const uint64_t*)(base + L.o_om);
  v.chain_norm = (const int32_t*)(base + L.o_cn);
  v.tab = (const DTable*)(base + L.o_tab);
  v.par = (const uint64_t*)(base + L.o_par);
  v.pidx = (const uint2*)(base + L.o_pidx);
  v.cls = (const DClass*)(base + L.o_cls);
  v.fidx = (const uint32_t*)(base + L.o_fidx);
  v.finc = (const uint32_t*)(base + L.o_finc);
  v.fcoord = (const uint64_t*)(base + L.o_fco);
  v.seg = (const DSeg*)(base + L.o_seg);
  v.sb = (const DSBatch*)(base + L.o_sb);
  v.rows = (const uint32_t*)(base + L.o_row);
  v.sl_par = L.sl_par;
  v.sl_rb = L.sl_rb;
  v.dmap_off = (const int32_t*)(base + L.o_dmo);
  v.dmap_idx = (const int32_t*)(base + L.o_dmi);
  v.omap_off = (const int32_t*)(base + L.o_omo);
  v.omap_idx = (const int32_t*)(base + L.o_omi);
  v.chain_float = (const int32_t*)(base + L.o_cf);
  v.tconst = (const DConst*)(base + L.o_tc);
  v.dmask = (const uint64_t*)(base + L.o_dmk);
  v.omask2 = (const uint64_t*)(base + L.o_omk);
  v.dcst = (const int32_t*)(base + L.o_dcs);
  v.ocst = (const int32_t*)(base + L.o_ocs);
  v.ffidx = (const uint32_t*)(base + L.o_ffi);
  v.ffang = (const double*)(base + L.o_ffa);
  return v;
}

const DeviceTables& tables_of(const Program& p) {
  if (!p.devtab) fail(TSIM_ERR_INTERNAL, "program has no device tables");
  if (p.devtab->status != TSIM_OK) fail(p.devtab->status, p.devtab->message);
  return *p.devtab;
}

DeviceProgram* upload(const Program& p) {
  const DeviceTables& T = tables_of(p);
  auto* d = new DeviceProgram();
  TSIM_CUDA(cudaGetDevice(&d->device));
  cudaError_t e = cudaMalloc(&d->blob, std::max<size_t>(T.blob.size(), 256));
  if (e != cudaSuccess) {
    delete d;
    fail(TSIM_ERR_OOM, std::string("cudaMalloc of program tables: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(d->blob, T.blob.data(), T.blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d->blob);
    delete d;
    fail(TSIM_ERR_CUDA, std::string("cudaMemcpy of program tables: ") + cudaGetErrorString(e));
  }
  d->v = make_view((const unsigned char*)d->blob, T.layout, p);
  d->v.status = status_word(d->device);
  return d;
}

const DevView& ensure_uploaded(const Program& p) {
  int cur = -1;
  TSIM_CUDA(cudaGetDevice(&cur));
  auto& slot = const_cast<Program&>(p).dev;
  if (slot && slot->device != cur) {
    device_release(slot);
    slot = nullptr;
  }
  if (!slot) slot = upload(p);
  return slot->v;
}

// one program's sampling launch, dispatched on the padded width of X
cudaError_t launch(const LaunchArgs& a) {
  switch (a.v.W) {
    case 1: return launch_sample<1>(a);
    case 2: return launch_sample<2>(a);
    case 4: return launch_sample<4>(a);
    case 8: return launch_sample<8>(a);
    case 16: return launch_sample<16>(a);
    case 32: return launch_sample<32>(a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch(const DevView& v, cudaStream_t s, uint64_t seed, uint64_t off, uint64_t shots, uint64_t* meas,
                   uint64_t* det, uint64_t* obs, uint8_t* acc) {
  LaunchArgs a{};
  a.v = v;
  a.stream = s;
  a.seed = seed;
  a.shot_offset = off;
  a.shots = shots;
  a.meas = meas;
  a.det = det;
  a.obs = obs;
  a.accept = acc;
  return launch(a);
}

}  // namespace


// Host emulation of the warp-cooperative evaluation of a sliced table, read
// from the packed tables exactly as the kernel reads them: 32 per-shot
// vectors X at once (bit s of every word belongs to vector s).  Returns the
// exact value of table t for each vector.
std::vector<ZW> emulate_sliced_table(const Program& p, const DeviceTables& T, int t,
                                     const std::vector<std::vector<uint64_t>>& xs) {
  const DeviceLayout& L = T.layout;
  const unsigned char* b = T.blob.data();
  const DTable& tb = ((const DTable*)(b + L.o_tab))[t];
  const DSeg* seg = (const DSeg*)(b + L.o_seg);
  const DSBatch* sbv = (const DSBatch*)(b + L.o_sb);
  const uint32_t* rows = (const uint32_t*)(b + L.o_row);
  const uint64_t* par = (const uint64_t*)(b + L.o_par);
  const uint2* pidx = (const uint2*)(b + L.o_pidx);
  const int W = L.W;
  std::vector<ZW> val(32);
  std::vector<uint32_t> Xs((size_t)64 * W, 0);
  for (int sh = 0; sh < 32; ++sh)
    for (int i = 0; i < 64 * W; ++i)
      if ((xs[(size_t)sh][(size_t)i >> 6] >> (i & 63)) & 1) Xs[(size_t)i] |= 1u << sh;
  for (int g = 0; g < tb.n_sb; ++g) {
    const DSeg& sg = seg[tb.sb_off + g];
    std::vector<uint32_t> Par(sg.n_par, 0);
    for (uint32_t q = 0; q < sg.n_par; ++q) {
      uint32_t acc = 0;
      for (int w = 0; w < W; ++w)
        for (int bit = 0; bit < 64; ++bit)
          if ((par[((size_t)sg.par_off + q) * W + (size_t)w] >> bit) & 1) acc ^= Xs[(size_t)(64 * w + bit)];
      // the kernel's form: four or eight named X bits, or the mask
      const uint2 ix = pidx[(size_t)sg.par_off + q];
      if (ix.x != kSlWalk) {
        uint32_t acc8 = 0;
        for (int k = 0; k < (sg.k8 ? 8 : 4); ++k) acc8 ^= Xs[(size_t)((((k < 4) ? ix.x : ix.y) >> (8 * (k & 3))) & 0xFF)];
        if (acc8 != acc) fail(TSIM_ERR_INTERNAL, "a parity's bit indices differ from its mask");
      }
      Par[q] = q == kSlOnes ? 0xFFFFFFFFu : acc;
    }
    auto word = [&](uint32_t off) {
      if (off % 4 || off / 4 >= sg.n_par) fail(TSIM_ERR_INTERNAL, "sliced row outside its segment's parity words");
      return Par[off / 4];
    };
    for (uint32_t bi = 0; bi < sg.n_sb; ++bi) {
      const DSBatch& B = sbv[sg.sb_off + bi];
      uint32_t J0[32], J1[32], J2[32], Z[32];
      for (int l = 0; l < 32; ++l) {
        J0[l] = 0u - ((B.j0m[0] >> l) & 1u);
        J1[l] = 0u - ((B.j0m[1] >> l) & 1u);
        J2[l] = 0u - ((B.j0m[2] >> l) & 1u);
        Z[l] = 0u - ((~B.valid >> l) & 1u);
      }
      size_t at = B.row_off;
      for (int c = 0; c < kSlCodes; ++c) {
        const uint32_t n = B.cnt[c];
        if (n % 4) fail(TSIM_ERR_INTERNAL, "sliced rows not in groups of 4");
        for (uint32_t k = 0; k < n; ++k)
          for (int l = 0; l < 32; ++l) {
            const uint32_t r = rows[at + (size_t)(k / 4) * 128 + (size_t)l * 4 + (k % 4)];
            const uint32_t a = c == SL_XOR4AB ? word(r & 0xFFFFu) & word(r >> 16) : word(r);
            auto add = [&](uint32_t m, int times) {  // J += times * m (mod 8), one plane step at a time
              for (int i = 0; i < times; ++i) {
                const uint32_t c0 = J0[l] & m;
                J0[l] ^= m;
                const uint32_t c1 = J1[l] & c0;
                J1[l] ^= c0;
                J2[l] ^= c1;
              }
            };
            switch (c) {
              case SL_XOR4: case SL_XOR4AB: add(a, 4); break;
              case SL_ADD2: add(a, 2); break;
              case SL_ADD6: add(a, 6); break;
              case SL_ADD1: add(a, 1); break;
              case SL_ZERO: Z[l] |= a; break;
              case SL_ZEROC: Z[l] |= ~a; break;
            }
          }
        at += (size_t)n * 32;
      }
      for (int sh = 0; sh < 32; ++sh)
        for (int l = 0; l < 32; ++l) {
          if ((Z[l] >> sh) & 1) continue;
          const int J = (int)((J0[l] >> sh) & 1) | (int)(((J1[l] >> sh) & 1) << 1) | (int)(((J2[l] >> sh) & 1) << 2);
          ZW term = ZW::omega(J);
          term.k = B.d + tb.base;
          val[(size_t)sh] = zw_add(val[(size_t)sh], term);
        }
    }
  }
  return val;
}

void selftest_sliced(const Program& p, uint64_t seed, int rounds) {
  const DeviceTables& T = tables_of(p);
  const int W = T.layout.W;
  uint64_t st = seed ^ 0x5EED5EEDull;
  auto rnd = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (size_t t = 0; t < p.tables.size(); ++t) {
    if (T.layout.table_mode[t] != TAB_SLICED) continue;
    for (int r = 0; r < rounds; ++r) {
      std::vector<std::vector<uint64_t>> xs(32, std::vector<uint64_t>((size_t)W, 0));
      for (auto& x : xs)
        for (int i = 0; i < p.nx; ++i)  // X bits beyond n_x stay zero, as on the device
          if (rnd() & 1) x[(size_t)i >> 6] |= 1ull << (i & 63);
      const std::vector<ZW> got = emulate_sliced_table(p, T, (int)t, xs);
      for (int sh = 0; sh < 32; ++sh) {
        ZW want = eval_table_host(p, (int)t, xs[(size_t)sh].data());
        for (auto& c : want.c) c = -c;
        if (!zw_add(got[(size_t)sh], want).zero())
          fail(TSIM_ERR_INTERNAL, "sliced table " + std::to_string(t) + " differs from the exact evaluation");
      }
    }
  }
}

void prepare_device_tables(Program& p, int64_t sliced_min, int stage_rows, int seg_par) {
  auto* t = new DeviceTables();
  t->sliced_min = sliced_min;
  t->stage_rows = stage_rows;
  t->seg_par = seg_par;
  try {
    pack(p, *t, sliced_min, stage_rows < 0 ? kDefaultStageRows : stage_rows,
         seg_par <= 0 ? kDefaultSegmentParities : std::max(seg_par, 16));
  } catch (const PackError& e) {
    t->status = e.st;
    t->message = e.msg;
    t->blob.clear();
  }
  delete p.devtab;
  p.devtab = t;
}

void device_sample(const Program& p, const SampleArgs& a, void* stream) {
  if (p.mode == TSIM_MODE_DETECTORS && a.meas) fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  tables_of(p);  // report a program that cannot run on the device before any CUDA call
  if (a.shots == 0) return;
  if (a.shots > 0x7FFFFFFFull * 32) fail(TSIM_ERR_ARG, "too many shots for one launch");
  const DevView& v = ensure_uploaded(p);
  cudaError_t e = launch(v, (cudaStream_t)stream, a.seed, a.shot_offset, a.shots, a.meas, a.det, a.obs, a.accept);
  if (e != cudaSuccess) fail(TSIM_ERR_CUDA, std::string("sampling kernel launch: ") + cudaGetErrorString(e));
}

// ----------------------------------------------------------- batch plans
// Programs of a batch fall in groups by whether they have sliced tables and
// by their X width: each group is one persistent launch with its own
// register budget (the kernels with sliced tables keep fewer warps
// resident) and its own width (a narrow program does not pay for the
// widest one's X).
struct BatchGroup {
  int off = 0, n = 0;       // programs [off, off + n) of the plan's (reordered) list
  int wmax = 1, sl_par = 0, sl_rb = 0;
  uint64_t total_items = 0;
  uint64_t* d_item_start = nullptr;   // n + 1 entries
  unsigned long long* d_counter = nullptr;
};

struct BatchPlan {
  int device = -1, n = 0, sms = 1;
  uint32_t sb = 128;        // shots per work item
  int blocks_per_sm = 8;
  static constexpr int kGroups = 12;  // (sliced tables or not) x (X width 1, 2, 4, ..., 32)
  BatchGroup grp[kGroups];
  std::vector<BatchProg> h_progs;  // group 0 first, then group 1, ...
  unsigned char* dmem = nullptr;
  BatchProg* d_progs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float tuned_ms = 0;
  int form = 0;  // 0: persistent launches over the work items; 1: each program's own launch
  uint64_t total_items() const {
    uint64_t t = 0;
    for (const BatchGroup& g : grp) t += g.total_items;
    return t;
  }
  int wmax() const {
    int w = 1;
    for (const BatchGroup& g : grp)
      if (g.n) w = std::max(w, g.wmax);
    return w;
  }
};

namespace {

void plan_items(BatchPlan& b, cudaStream_t s) {
  for (BatchGroup& g : b.grp) {
    std::vector<uint64_t> start((size_t)g.n + 1, 0);
    for (int i = 0; i < g.n; ++i)
      start[(size_t)i + 1] = start[(size_t)i] + (b.h_progs[(size_t)(g.off + i)].shots + b.sb - 1) / b.sb;
    g.total_items = start[(size_t)g.n];
    TSIM_CUDA(cudaMemcpyAsync(g.d_item_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice, s));
  }
  TSIM_CUDA(cudaStreamSynchronize(s));
}


cudaError_t launch_batch(const BatchPlan& b, cudaStream_t s) {
  if (b.form == 1) {  // the programs' own sampling launches, one after another
    for (const BatchProg& p : b.h_progs) {
      if (!p.shots) continue;
      cudaError_t e = launch(p.v, s, p.seed, p.shot_offset, p.shots, p.meas, p.det, p.obs, p.accept);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (const BatchGroup& g : b.grp) {
    if (!g.total_items) continue;
    cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const uint64_t want = (uint64_t)b.sms * (uint64_t)b.blocks_per_sm;
    BatchLaunchArgs a{};
    a.progs = b.d_progs + g.off;
    a.n = g.n;
    a.item_start = g.d_item_start;
    a.total_items = g.total_items;
    a.sb = b.sb;
    a.counter = g.d_counter;
    a.sl_par = g.sl_par;
    a.sl_rb = g.sl_rb;
    a.stream = s;
    a.grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, g.total_items));
    switch (g.wmax) {
      case 1: e = launch_batch_group<1>(a); break;
      case 2: e = launch_batch_group<2>(a); break;
      case 4: e = launch_batch_group<4>(a); break;
      case 8: e = launch_batch_group<8>(a); break;
      case 16: e = launch_batch_group<16>(a); break;
      case 32: e = launch_batch_group<32>(a); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

BatchPlan* batch_create(const Program* const* progs, int n, const SampleArgs* args, int autotune) {
  auto b = std::make_unique<BatchPlan>();
  b->n = n;
  TSIM_CUDA(cudaGetDevice(&b->device));
  TSIM_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
  std::vector<BatchProg> per_group[BatchPlan::kGroups];
  for (int i = 0; i < n; ++i) {
    const Program& p = *progs[i];
    if (p.mode == TSIM_MODE_DETECTORS && args[i].meas)
      fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
    tables_of(p);
    BatchProg bp{};
    bp.v = ensure_uploaded(p);
    bp.shots = args[i].shots;
    bp.seed = args[i].seed;
    bp.shot_offset = args[i].shot_offset;
    bp.meas = args[i].meas;
    bp.det = args[i].det;
    bp.obs = args[i].obs;
    bp.accept = args[i].accept;
    int wl = 0;
    while ((1 << wl) < bp.v.W) ++wl;
    if (wl > 5) fail(TSIM_ERR_ARG, "X wider than 32 words");
    const int gi = (bp.v.sl_par > 0 ? 6 : 0) + wl;
    BatchGroup& g = b->grp[gi];
    g.wmax = std::max(g.wmax, bp.v.W);
    g.sl_par = std::max(g.sl_par, bp.v.sl_par);
    g.sl_rb = std::max(g.sl_rb, bp.v.sl_rb);
    per_group[gi].push_back(bp);
  }
  {
    int off = 0;
    for (int gi = 0; gi < BatchPlan::kGroups; ++gi) {
      b->grp[gi].off = off;
      b->grp[gi].n = (int)per_group[gi].size();
      off += b->grp[gi].n;
    }
  }
  for (const auto& v : per_group) b->h_progs.insert(b->h_progs.end(), v.begin(), v.end());
  const size_t bytes = (size_t)n * sizeof(BatchProg) + ((size_t)n + BatchPlan::kGroups) * 8 +
                       (size_t)BatchPlan::kGroups * 64;
  cudaError_t e = cudaMalloc(&b->dmem, bytes);
  if (e != cudaSuccess) fail(TSIM_ERR_OOM, std::string("cudaMalloc of the batch plan: ") + cudaGetErrorString(e));
  b->d_progs = (BatchProg*)b->dmem;
  {
    uint64_t* starts = (uint64_t*)(b->dmem + (size_t)n * sizeof(BatchProg));
    unsigned char* ctr = b->dmem + (size_t)n * sizeof(BatchProg) + ((size_t)n + BatchPlan::kGroups) * 8;
    for (int gi = 0; gi < BatchPlan::kGroups; ++gi) {
      b->grp[gi].d_item_start = starts + b->grp[gi].off + gi;  // n + 1 entries per group
      b->grp[gi].d_counter = (unsigned long long*)(ctr + 64 * gi);
    }
  }
  cudaStream_t s = nullptr;
  TSIM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct SD { cudaStream_t s; ~SD() { cudaStreamDestroy(s); } } sd{s};
  if (n) TSIM_CUDA(cudaMemcpyAsync(b->d_progs, b->h_progs.data(), (size_t)n * sizeof(BatchProg), cudaMemcpyHostToDevice, s));
  b->sb = 128;
  plan_items(*b, s);
  if (autotune == 2) b->form = 1;
  if (autotune == 1 && b->total_items()) {
    // shot-block size x resident blocks per SM: time every candidate twice on
    // the real batch (records are overwritten with identical values)
    cudaEvent_t e0, e1;
    TSIM_CUDA(cudaEventCreate(&e0));
    TSIM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    uint32_t best_sb = b->sb;
    int best_bps = b->blocks_per_sm;
    // work items of 32, 128 or 512 shots (one warp each)
    for (uint32_t sb : {32u, 128u, 512u}) {
      b->sb = sb;
      plan_items(*b, s);
      for (int bps : {4, 8, 16}) {
        b->blocks_per_sm = bps;
        float t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          TSIM_CUDA(cudaEventRecord(e0, s));
          TSIM_CUDA(launch_batch(*b, s));
          TSIM_CUDA(cudaEventRecord(e1, s));
          TSIM_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          TSIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          t = std::min(t, ms);
        }
        if (t < best) { best = t; best_sb = sb; best_bps = bps; }
      }
    }
    // the other launch form: every program's own kernel (few large programs
    // can run faster that way than through the persistent loop)
    {
      b->form = 1;
      float t = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        TSIM_CUDA(cudaEventRecord(e0, s));
        TSIM_CUDA(launch_batch(*b, s));
        TSIM_CUDA(cudaEventRecord(e1, s));
        TSIM_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        TSIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t = std::min(t, ms);
      }
      b->form = t < best ? 1 : 0;
      best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->sb = best_sb;
    b->blocks_per_sm = best_bps;
    b->tuned_ms = best;
    plan_items(*b, s);
  }
  // capture counter reset + persistent launch as one graph
  TSIM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch_batch(*b, s);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    fail(TSIM_ERR_CUDA, std::string("graph capture of the batched launch: ") +
                            cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  b->graph = g;
  TSIM_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  return b.release();
}

void batch_launch(BatchPlan* b, void* stream) {
  int cur = -1;
  TSIM_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) fail(TSIM_ERR_ARG, "batch launched on another device than it was created on");
  TSIM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

void batch_free(BatchPlan* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
}

void batch_info(const BatchPlan* b, int64_t out[7]) {
  out[0] = b->sb;
  out[1] = b->blocks_per_sm;
  out[2] = (int64_t)b->total_items();
  out[3] = b->exec ? 1 : 0;
  out[4] = b->wmax();
  out[5] = (int64_t)(b->tuned_ms * 1000.0f);
  out[6] = b->form;
}

void device_sample_batch(const Program* const* progs, int n, const SampleArgs* args, void* stream) {
  BatchPlan* b = batch_create(progs, n, args, 0);
  struct F { BatchPlan* b; ~F() { batch_free(b); } } f{b};
  batch_launch(b, stream);
  TSIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}


void device_sync(void* stream) {
  TSIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int dev = -1;
  TSIM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) fail(TSIM_ERR_ARG, "device index out of range");
  int* words[2] = {nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lock(g_status_mu);
    words[0] = g_status_dev[dev];
  }
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    words[1] = (int*)g_noalloc_dev[dev];
  }
  int st = 0;
  for (int* w : words) {
    if (!w) continue;
    int v = 0;
    TSIM_CUDA(cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
      st |= v;
      TSIM_CUDA(cudaMemset(w, 0, sizeof v));
    }
  }
  if (st) {
    if (st & ST_TIMEOUT) fail(TSIM_ERR_TIMEOUT, "device: a shared-memory staging copy did not complete in time");
    if (st & ST_ZERO_PROB) fail(TSIM_ERR_ZERO_PROB, "device: a sampled prefix had P_prev <= 0");
    if (st & ST_NOT_REAL) fail(TSIM_ERR_INTERNAL, "device: a marginal was not real");
    fail(TSIM_ERR_OVERFLOW_BOUND, "device: exact arithmetic overflow");
  }
}

void device_sample_debug(const Program& p, const SampleArgs& a, const uint64_t* dump_shots, int n_dump,
                         int64_t* h_dump, void* stream) {
  if (p.mode == TSIM_MODE_DETECTORS && a.meas) fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  const DeviceTables& T = tables_of(p);
  if (n_dump < 0 || (n_dump > 0 && (!dump_shots || !h_dump))) fail(TSIM_ERR_ARG, "bad dump arguments");
  if (a.shots == 0) return;
  if (a.shots > ((uint64_t)1 << 31)) fail(TSIM_ERR_ARG, "debug launches are limited to 2^31 shots");
  std::vector<int32_t> row(a.shots, -1);
  for (int k = 0; k < n_dump; ++k) {
    if (dump_shots[k] >= a.shots || row[(size_t)dump_shots[k]] >= 0) fail(TSIM_ERR_ARG, "dump shots must be distinct and inside the launch");
    row[(size_t)dump_shots[k]] = k;
  }
  const DevView& v = ensure_uploaded(p);
  const int evals = (int)p.chain_norm.size() + p.nr;
  const int wdev = T.layout.W;
  const int stride = evals * (kDumpHead + wdev);
  struct Buf {
    void* p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
  } drow, ddump;
  TSIM_CUDA(cudaMalloc(&drow.p, row.size() * sizeof(int32_t)));
  TSIM_CUDA(cudaMalloc(&ddump.p, std::max<size_t>(1, (size_t)n_dump * (size_t)stride) * sizeof(long long)));
  cudaStream_t s = (cudaStream_t)stream;
  TSIM_CUDA(cudaMemcpyAsync(drow.p, row.data(), row.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  TSIM_CUDA(cudaMemsetAsync(ddump.p, 0, std::max<size_t>(1, (size_t)n_dump * (size_t)stride) * sizeof(long long), s));
  LaunchArgs la{};
  la.v = v;
  la.stream = s;
  la.seed = a.seed;
  la.shot_offset = a.shot_offset;
  la.shots = a.shots;
  la.meas = a.meas;
  la.det = a.det;
  la.obs = a.obs;
  la.accept = a.accept;
  la.dump = (long long*)ddump.p;
  la.dump_row = (const int32_t*)drow.p;
  la.dump_stride = stride;
  cudaError_t e = launch(la);
  if (e != cudaSuccess) fail(TSIM_ERR_CUDA, std::string("debug sampling launch: ") + cudaGetErrorString(e));
  std::vector<long long> buf((size_t)n_dump * (size_t)stride);
  if (!buf.empty())
    TSIM_CUDA(cudaMemcpyAsync(buf.data(), ddump.p, buf.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
  TSIM_CUDA(cudaStreamSynchronize(s));
  // host layout: per shot, per evaluation, kDumpHead + x_words values
  const int wout = p.W;
  for (int k = 0; k < n_dump; ++k)
    for (int ev = 0; ev < evals; ++ev) {
      const long long* src = buf.data() + (size_t)k * stride + (size_t)ev * (kDumpHead + wdev);
      int64_t* dst = h_dump + ((size_t)k * evals + (size_t)ev) * (size_t)(kDumpHead + wout);
      for (int i = 0; i < kDumpHead + wout; ++i) dst[i] = src[i];
    }
}

void device_sample_noalloc(const Program& p, const SampleArgs& a, void* stream) {
  if (p.mode == TSIM_MODE_DETECTORS && a.meas) fail(TSIM_ERR_ARG, "measurement records requested from a detector-mode program");
  // the packed tables were built on the host when the program was compiled
  // or loaded; this call only copies them
  const DeviceTables& T = tables_of(p);
  if (T.layout.total > kNoAllocBytes - kNoAllocHead)
    fail(TSIM_ERR_ARG, "program tables exceed the 4 MiB maximum of tsim_sample_noalloc");
  if (a.shots == 0) return;
  if (a.shots > 0x7FFFFFFFull * 32) fail(TSIM_ERR_ARG, "too many shots for one launch");
  int dev = -1;
  TSIM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) fail(TSIM_ERR_ARG, "device index out of range");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TSIM_CUDA(cudaStreamIsCapturing(s, &cs));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    // with the device current: looked up again on every call that is not
    // being captured, so a device reset (which moves the array) is picked up
    void* ptr = nullptr;
    TSIM_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (!ptr) fail(TSIM_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch array returned NULL");
    g_noalloc_dev[dev] = ptr;
  } else if (!g_noalloc_dev[dev]) {
    fail(TSIM_ERR_ARG, "the first tsim_sample_noalloc call on a device must come before any stream capture");
  }
  unsigned char* base = (unsigned char*)g_noalloc_dev[dev];
  // every byte the kernel reads is rewritten here, so nothing stale from the
  // previous call survives; the status word is cleared by tsim_sync
  TSIM_CUDA(cudaMemcpyAsync(base + kNoAllocHead, T.blob.data(), T.layout.total, cudaMemcpyHostToDevice, s));
  DevView v = make_view(base + kNoAllocHead, T.layout, p);
  v.status = (int*)base;
  cudaError_t e = launch(v, s, a.seed, a.shot_offset, a.shots, a.meas, a.det, a.obs, a.accept);
  if (e != cudaSuccess) fail(TSIM_ERR_CUDA, std::string("sampling kernel launch: ") + cudaGetErrorString(e));
}

}  // namespace tsim
