/*
 * Oracle program evaluator: plain, slow, exact.  TEST INFRASTRUCTURE ONLY --
 * nothing in the product links or loads this file.
 *
 * Given a compiled program (read from its text file by the reader below, which
 * shares no code with the product), a 64-bit seed and a range of global shot
 * indices, it reproduces the sampler's output records by following the paper
 * step by step:
 *
 *   1. error mechanisms: every reduced noise channel draws one outcome from its
 *      joint distribution p(e_{i_k}..e_{i_{k+n}}) (Sec. "Detectors"), using one
 *      32-bit Philox4x32-10 word per channel and the channel's cumulative
 *      thresholds;
 *   2. f = T e mod 2 (Eq. detector_sampling): XOR of the column signatures of
 *      the fired outcomes;
 *   3. outputs in autoregressive order: a deterministic output is a GF(2)
 *      parity of (f, earlier outputs); a random output follows Algorithm 1
 *      (Appendix "Sampling from marginals"): P_prev starts at the chain's
 *      normalisation P, P_1 is the marginal with m_i = 1, the bit is drawn
 *      from Bernoulli(P_1 / P_prev) and P_prev is updated.  The diagrams of a
 *      chain are known up to the scalars that were discarded and that the
 *      normalisation P restores (Sec. "Observables"); with exact Clifford
 *      scalars that is a common phase w^j, so every table of the chain is
 *      multiplied by the w^-j that makes P real and positive;
 *   4. every marginal is P = sum_t c^t prod_k h(alpha_k, beta_k; a_k, b_k)
 *      with a_k = XOR_i u_ki f_i and b_k = XOR_i v_ki f_i (Eqs. parities,
 *      phase_pair, scalar_product), each factor computed from its defining
 *      formula as an element of Z[w] (w = e^{i pi/4}) -- never from a table;
 *   5. records: detector bits, observable bits (XOR of measurement bits in
 *      measurement mode, Eq. xor), bit-packed into uint64 rows, plus an
 *      acceptance flag (all detectors zero).
 *
 * Readings where the paper is silent (documented with the program format):
 *   - Philox4x32-10 (Salmon et al., SC'11): key = (seed lo, seed hi); counter =
 *     (shot lo, shot hi, stream, block); stream 0 feeds channel c from word
 *     c%4 of block c/4; stream 1 feeds output i from word i%4 of block i/4.
 *   - channel outcome = smallest o < n-1 with U < thr[o], else n-1.
 *   - Bernoulli rule, exact: bit = 1  iff  U * P_prev < 2^32 * P_1.
 *   - Geometric gaps (a program option; Sec. "Detectors" samples the gap
 *     between successive firing events from a geometric distribution, which
 *     takes O(p E) work instead of O(E)).  The channels are split into
 *     groups; group g lists its channels in order and a 32-bit Q_g no larger
 *     than the outcome-0 threshold of any member, so that every member fires
 *     with probability at most r_g = 1 - Q_g / 2^32.  Candidates are placed
 *     along the group as Bernoulli(r_g) trials: the number of non-candidates
 *     before the next candidate is the gap, with P(gap >= k) = T_k / 2^32,
 *     T_0 = 2^32 and T_k = floor(T_{k-1} Q_g / 2^32) (a geometric law with
 *     ratio Q_g / 2^32, each step rounded down).  At a candidate channel c a
 *     second word V is mapped onto [Q_g, 2^32) by V' = Q_g +
 *     floor(V (2^32 - Q_g) / 2^32), and the channel's own threshold rule is
 *     applied to V' (so the candidate is rejected, outcome 0, with
 *     probability (thr_c[0] - Q_g) / (2^32 - Q_g)).  All words of a shot come
 *     from stream 2, in the order they are used: word j is word j%4 of block
 *     j/4; groups in program order; within a group, while channels remain, a
 *     gap word, and when it places a candidate, that candidate's word V.
 *
 * Arbitrary rotations (R_X, R_Y, R_Z, U3 at angles that are not multiples of
 * pi/4) leave the exact ring: their tables carry a constant phase
 * e^(i pi phase) per term and factors e^(i pi t a) (Table "Types of
 * parameterized phase terms" with an arbitrary angle).  A chain with such a
 * table is evaluated in double-precision complex arithmetic: the chain's
 * common phase is that of its normalisation z_n, so P_prev = |z_n| and a
 * marginal z_1 gives P_1 = Re(z_1 conj(z_n)) / |z_n|.  The Bernoulli draw
 * rounds the ratio P_1 / P_prev to the nearest FP32 value q and sets the bit
 * iff U < q 2^32 (the decision both implementations take in the same
 * precision, whatever the order of their sums).
 *
 * Arithmetic: __int128 with every operation overflow-checked; an overflow or
 * a non-real marginal aborts the call with an error message rather than
 * returning a wrong bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

static __thread char g_err[512];

static int fail(const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return -1;
}

const char* oracle_last_error(void) { return g_err; }

/* ------------------------------------------------------------------ Philox */
/* Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror, Shaw (SC'11):
 * round: (hi0,lo0) = M0*x0, (hi1,lo1) = M1*x2,
 *        x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); key bumped by the
 *        Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * x0, p1 = (uint64_t)M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t philox_word(uint64_t seed, uint64_t shot, uint32_t stream, uint32_t index) {
  uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), stream, index >> 2};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  oracle_philox4x32_10(ctr, key, out);
  return out[index & 3];
}

/* --------------------------------------------------------- checked int128 */
static int g_ovf;
static i128 add_(i128 a, i128 b) { i128 r; if (__builtin_add_overflow(a, b, &r)) g_ovf = 1; return r; }
static i128 sub_(i128 a, i128 b) { i128 r; if (__builtin_sub_overflow(a, b, &r)) g_ovf = 1; return r; }
static i128 mul_(i128 a, i128 b) { i128 r; if (__builtin_mul_overflow(a, b, &r)) g_ovf = 1; return r; }
static i128 shl_(i128 a, int s) {
  for (int i = 0; i < s; ++i) a = mul_(a, 2);
  return a;
}

/* ----------------------------------------------------------- Z[w] values */
/* value = (c0 + c1 w + c2 w^2 + c3 w^3) * sqrt2^k,  w^4 = -1 */
typedef struct { i128 c[4]; int k; } zw;

static zw zw_zero(void) { zw z; memset(&z, 0, sizeof z); return z; }

static zw zw_omega(int j) {  /* w^j */
  zw z = zw_zero();
  j = ((j % 8) + 8) % 8;
  if (j < 4) z.c[j] = 1; else z.c[j - 4] = -1;
  return z;
}

static int zw_is_zero(const zw* a) { return !(a->c[0] || a->c[1] || a->c[2] || a->c[3]); }

static zw zw_mul(zw a, zw b) {
  zw r = zw_zero();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      i128 p = mul_(a.c[i], b.c[j]);
      int n = i + j;
      if (n >= 4) r.c[n - 4] = sub_(r.c[n - 4], p);
      else r.c[n] = add_(r.c[n], p);
    }
  r.k = a.k + b.k;
  return r;
}

static zw zw_times_sqrt2(zw a) {  /* sqrt2 = w - w^3 */
  zw s = zw_zero();
  s.c[1] = 1; s.c[3] = -1;
  zw r = zw_mul(a, s);
  r.k = a.k;
  return r;
}

static zw zw_add(zw a, zw b) {
  if (zw_is_zero(&a)) return b;
  if (zw_is_zero(&b)) return a;
  /* bring both to the smaller exponent */
  while (a.k > b.k) { a = zw_times_sqrt2(a); a.k -= 1; }
  while (b.k > a.k) { b = zw_times_sqrt2(b); b.k -= 1; }
  zw r;
  for (int i = 0; i < 4; ++i) r.c[i] = add_(a.c[i], b.c[i]);
  r.k = a.k;
  return r;
}

/* ------------------------------------------------------------ real values */
/* (A + B sqrt2) * 2^e */
typedef struct { i128 A, B; int e; } rv;

static int zw_to_real(const zw* z, rv* out) {
  if (z->c[2] != 0 || add_(z->c[1], z->c[3]) != 0) return fail("marginal is not real");
  /* Re = c0 + (c1 - c3)/sqrt2 = (2 c0 + (c1 - c3) sqrt2) / 2 ; times sqrt2^k */
  i128 A = mul_(2, z->c[0]), B = sub_(z->c[1], z->c[3]);
  int k = z->k - 2;
  if (k & 1) {  /* (A + B sqrt2) sqrt2 = 2B + A sqrt2 */
    i128 t = A;
    A = mul_(2, B);
    B = t;
    k -= 1;
  }
  out->A = A; out->B = B; out->e = k / 2;
  if (k % 2) return fail("internal parity error");
  return 0;
}

static void rv_align(rv* a, rv* b) {
  if (a->A == 0 && a->B == 0) { a->e = b->e; return; }
  if (b->A == 0 && b->B == 0) { b->e = a->e; return; }
  while (a->e > b->e) { a->A = shl_(a->A, 1); a->B = shl_(a->B, 1); a->e -= 1; }
  while (b->e > a->e) { b->A = shl_(b->A, 1); b->B = shl_(b->B, 1); b->e -= 1; }
}

/* unsigned 128 x 128 -> 256 as four 64-bit limbs, little endian */
static void mul256(u128 a, u128 b, uint64_t r[4]) {
  uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
  u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  r[0] = (uint64_t)p00;
  r[1] = (uint64_t)mid;
  u128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
  r[2] = (uint64_t)hi;
  r[3] = (uint64_t)((hi >> 64) + (p11 >> 64));
}

static int cmp256(const uint64_t a[4], const uint64_t b[4]) {
  for (int i = 3; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}

static u128 uabs(i128 x) { return x < 0 ? (u128)(-(x + 1)) + 1 : (u128)x; }

/* exact sign of X + Y sqrt2 */
static int sign_xy(i128 X, i128 Y) {
  if (X >= 0 && Y >= 0) return (X == 0 && Y == 0) ? 0 : 1;
  if (X <= 0 && Y <= 0) return -1;
  uint64_t x2[4], y2[4];
  u128 ax = uabs(X), ay = uabs(Y);
  mul256(ax, ax, x2);
  mul256(ay, ay, y2);
  /* 2 * y2 */
  uint64_t carry = 0;
  for (int i = 0; i < 4; ++i) {
    uint64_t v = y2[i];
    y2[i] = (v << 1) | carry;
    carry = v >> 63;
  }
  if (carry) { g_ovf = 1; }
  int c = cmp256(x2, y2);  /* sign of X^2 - 2 Y^2 */
  if (X > 0) return c > 0 ? 1 : -1;   /* Y < 0 */
  return c < 0 ? 1 : -1;              /* X < 0 < Y */
}

/* ---------------------------------------------------------- the program */
typedef struct {
  int kind, alpha, beta;
  double t;  /* kind 4: e^(i pi t a) */
  uint64_t* u; uint64_t* v;
} factor;
typedef struct { int s0, j0, nf; double fph; factor* f; } term;
typedef struct { int nt, flt; term* t; } table;
typedef struct { int is_random; uint64_t* mask; int cst; int xbit, chain, table; } output;
typedef struct { int n_out; uint32_t* thr; uint64_t* sig; } channel;
/* geometric-gap group: members in order, Q, and T_1..T_n (T[k], T[0] unused) */
typedef struct { uint32_t Q; int n; int* member; uint32_t* T; } group;

struct oracle_prog {
  int mode;  /* 0 detectors, 1 measurements */
  int nx, W, nf, nr, nmeas, ndet, nobs;
  int n_out; output* out;
  int n_chains; int* chain_norm;
  int* chain_float;  /* the chain has a table with arbitrary phases */
  int n_ch; channel* ch;
  int noise_mode;  /* 0 one word per channel, 1 geometric gaps */
  int n_groups; group* groups;
  int n_tab; table* tab;
  int n_detmap; int* detmap_n; int** detmap;
  int n_obsmap; int* obsmap_n; int** obsmap;
};

static int read_hex_words(FILE* f, int W, uint64_t* dst) {
  for (int i = 0; i < W; ++i) {
    unsigned long long v;
    if (fscanf(f, "%llx", &v) != 1) return -1;
    dst[i] = (uint64_t)v;
  }
  return 0;
}

static int expect(FILE* f, const char* word) {
  char buf[64];
  if (fscanf(f, "%63s", buf) != 1) return -1;
  return strcmp(buf, word) == 0 ? 0 : -1;
}

void oracle_free(struct oracle_prog* p);

struct oracle_prog* oracle_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) { fail("cannot open program file"); return NULL; }
  struct oracle_prog* p = calloc(1, sizeof *p);
  char mode[32];
  int ver;
  if (expect(f, "TSIMPROG") || fscanf(f, "%d", &ver) != 1 || ver != 2) goto bad;
  if (expect(f, "mode") || fscanf(f, "%31s", mode) != 1) goto bad;
  p->mode = strcmp(mode, "measurements") == 0;
  if (expect(f, "nx") || fscanf(f, "%d", &p->nx) != 1) goto bad;
  if (expect(f, "words") || fscanf(f, "%d", &p->W) != 1) goto bad;
  if (expect(f, "nf") || fscanf(f, "%d", &p->nf) != 1) goto bad;
  if (expect(f, "nr") || fscanf(f, "%d", &p->nr) != 1) goto bad;
  if (expect(f, "nmeas") || fscanf(f, "%d", &p->nmeas) != 1) goto bad;
  if (expect(f, "ndet") || fscanf(f, "%d", &p->ndet) != 1) goto bad;
  if (expect(f, "nobs") || fscanf(f, "%d", &p->nobs) != 1) goto bad;
  int W = p->W;
  if (W < 1 || W > 64) goto bad;
  if (expect(f, "outputs") || fscanf(f, "%d", &p->n_out) != 1) goto bad;
  p->out = calloc((size_t)p->n_out + 1, sizeof(output));
  for (int i = 0; i < p->n_out; ++i) {
    char tag[8];
    if (fscanf(f, "%7s", tag) != 1) goto bad;
    output* o = &p->out[i];
    if (strcmp(tag, "D") == 0) {
      o->mask = calloc(W, 8);
      if (read_hex_words(f, W, o->mask) || fscanf(f, "%d", &o->cst) != 1) goto bad;
    } else if (strcmp(tag, "R") == 0) {
      o->is_random = 1;
      if (fscanf(f, "%d %d %d", &o->xbit, &o->chain, &o->table) != 3) goto bad;
    } else goto bad;
  }
  if (expect(f, "chains") || fscanf(f, "%d", &p->n_chains) != 1) goto bad;
  p->chain_norm = calloc((size_t)p->n_chains + 1, sizeof(int));
  for (int i = 0; i < p->n_chains; ++i)
    if (expect(f, "C") || fscanf(f, "%d", &p->chain_norm[i]) != 1) goto bad;
  if (expect(f, "channels") || fscanf(f, "%d", &p->n_ch) != 1) goto bad;
  p->ch = calloc((size_t)p->n_ch + 1, sizeof(channel));
  for (int c = 0; c < p->n_ch; ++c) {
    channel* ch = &p->ch[c];
    if (expect(f, "K") || fscanf(f, "%d", &ch->n_out) != 1 || ch->n_out < 1) goto bad;
    ch->thr = calloc((size_t)ch->n_out, sizeof(uint32_t));
    for (int o = 0; o + 1 < ch->n_out; ++o) {
      unsigned long long t;
      if (fscanf(f, "%llu", &t) != 1) goto bad;
      ch->thr[o] = (uint32_t)t;
    }
    ch->sig = calloc((size_t)ch->n_out * W, 8);
    for (int o = 0; o < ch->n_out; ++o)
      if (expect(f, "S") || read_hex_words(f, W, ch->sig + (size_t)o * W)) goto bad;
  }
  if (expect(f, "noise") || fscanf(f, "%d %d", &p->noise_mode, &p->n_groups) != 2) goto bad;
  if (p->noise_mode < 0 || p->noise_mode > 1 || p->n_groups < 0) goto bad;
  if (p->noise_mode == 0 && p->n_groups != 0) goto bad;
  p->groups = calloc((size_t)p->n_groups + 1, sizeof(group));
  {
    /* every channel that can fire belongs to exactly one group */
    int* seen = calloc((size_t)p->n_ch + 1, sizeof(int));
    int okg = 1;
    for (int g = 0; g < p->n_groups && okg; ++g) {
      group* G = &p->groups[g];
      unsigned long long q;
      if (expect(f, "G") || fscanf(f, "%llu %d", &q, &G->n) != 2 || q > 0xFFFFFFFFull || G->n < 1) { okg = 0; break; }
      G->Q = (uint32_t)q;
      G->member = calloc((size_t)G->n, sizeof(int));
      G->T = calloc((size_t)G->n + 1, sizeof(uint32_t));
      for (int k = 0; k < G->n; ++k) {
        int c;
        if (fscanf(f, "%d", &c) != 1 || c < 0 || c >= p->n_ch || seen[c]) { okg = 0; break; }
        seen[c] = 1;
        /* Q_g must not exceed the member's outcome-0 threshold */
        if (p->ch[c].n_out < 2 || p->ch[c].thr[0] < G->Q) { okg = 0; break; }
        G->member[k] = c;
      }
      /* T_k = floor(T_{k-1} Q / 2^32), T_0 = 2^32 */
      uint64_t t = (uint64_t)1 << 32;
      for (int k = 1; okg && k <= G->n; ++k) {
        t = (t * (uint64_t)G->Q) >> 32;
        G->T[k] = (uint32_t)t;
      }
    }
    for (int c = 0; okg && p->noise_mode == 1 && c < p->n_ch; ++c)
      if (p->ch[c].n_out >= 2 && !seen[c]) okg = 0;
    free(seen);
    if (!okg) goto bad;
  }
  if (expect(f, "tables") || fscanf(f, "%d", &p->n_tab) != 1) goto bad;
  p->tab = calloc((size_t)p->n_tab + 1, sizeof(table));
  for (int ti = 0; ti < p->n_tab; ++ti) {
    table* tb = &p->tab[ti];
    if (expect(f, "T") || fscanf(f, "%d %d", &tb->nt, &tb->flt) != 2 || tb->flt < 0 || tb->flt > 1) goto bad;
    tb->t = calloc((size_t)tb->nt + 1, sizeof(term));
    for (int t = 0; t < tb->nt; ++t) {
      term* tm = &tb->t[t];
      if (expect(f, "t") || fscanf(f, "%d %d %d", &tm->s0, &tm->j0, &tm->nf) != 3) goto bad;
      if (tb->flt && fscanf(f, "%lf", &tm->fph) != 1) goto bad;
      tm->f = calloc((size_t)tm->nf + 1, sizeof(factor));
      for (int k = 0; k < tm->nf; ++k) {
        factor* fc = &tm->f[k];
        if (expect(f, "f") || fscanf(f, "%d %d %d", &fc->kind, &fc->alpha, &fc->beta) != 3) goto bad;
        fc->u = calloc(W, 8);
        fc->v = calloc(W, 8);
        if (read_hex_words(f, W, fc->u) || read_hex_words(f, W, fc->v)) goto bad;
        if (fc->kind == 4 && (!tb->flt || fscanf(f, "%lf", &fc->t) != 1)) goto bad;
      }
    }
  }
  if (expect(f, "detmap")) goto bad;
  int nd;
  if (fscanf(f, "%d", &nd) != 1) goto bad;
  p->n_detmap = nd;
  p->detmap_n = calloc((size_t)nd + 1, sizeof(int));
  p->detmap = calloc((size_t)nd + 1, sizeof(int*));
  for (int d = 0; d < nd; ++d) {
    if (expect(f, "M") || fscanf(f, "%d", &p->detmap_n[d]) != 1) goto bad;
    p->detmap[d] = calloc((size_t)p->detmap_n[d] + 1, sizeof(int));
    for (int j = 0; j < p->detmap_n[d]; ++j)
      if (fscanf(f, "%d", &p->detmap[d][j]) != 1) goto bad;
  }
  if (expect(f, "obsmap")) goto bad;
  int no;
  if (fscanf(f, "%d", &no) != 1) goto bad;
  p->n_obsmap = no;
  p->obsmap_n = calloc((size_t)no + 1, sizeof(int));
  p->obsmap = calloc((size_t)no + 1, sizeof(int*));
  for (int d = 0; d < no; ++d) {
    if (expect(f, "M") || fscanf(f, "%d", &p->obsmap_n[d]) != 1) goto bad;
    p->obsmap[d] = calloc((size_t)p->obsmap_n[d] + 1, sizeof(int));
    for (int j = 0; j < p->obsmap_n[d]; ++j)
      if (fscanf(f, "%d", &p->obsmap[d][j]) != 1) goto bad;
  }
  if (p->mode == 1 && (nd != p->ndet || no != p->nobs)) goto bad;
  /* a chain is evaluated in floating point when any of its tables is */
  p->chain_float = calloc((size_t)p->n_chains + 1, sizeof(int));
  for (int c = 0; c < p->n_chains; ++c) {
    if (p->chain_norm[c] < 0 || p->chain_norm[c] >= p->n_tab) goto bad;
    p->chain_float[c] = p->tab[p->chain_norm[c]].flt;
  }
  for (int i = 0; i < p->n_out; ++i) {
    const output* o = &p->out[i];
    if (!o->is_random) continue;
    if (o->chain < 0 || o->chain >= p->n_chains || o->table < 0 || o->table >= p->n_tab) goto bad;
    if (p->tab[o->table].flt) p->chain_float[o->chain] = 1;
  }
  /* the raw-channel section that follows is verification data; not needed */
  fclose(f);
  return p;
bad:
  fclose(f);
  oracle_free(p);
  fail("malformed program file");
  return NULL;
}

void oracle_free(struct oracle_prog* p) {
  if (!p) return;
  for (int i = 0; p->out && i < p->n_out; ++i) free(p->out[i].mask);
  free(p->out);
  free(p->chain_norm);
  free(p->chain_float);
  for (int c = 0; p->ch && c < p->n_ch; ++c) { free(p->ch[c].thr); free(p->ch[c].sig); }
  free(p->ch);
  for (int g = 0; p->groups && g < p->n_groups; ++g) { free(p->groups[g].member); free(p->groups[g].T); }
  free(p->groups);
  for (int ti = 0; p->tab && ti < p->n_tab; ++ti) {
    table* tb = &p->tab[ti];
    for (int t = 0; tb->t && t < tb->nt; ++t) {
      for (int k = 0; k < tb->t[t].nf; ++k) { free(tb->t[t].f[k].u); free(tb->t[t].f[k].v); }
      free(tb->t[t].f);
    }
    free(tb->t);
  }
  free(p->tab);
  if (p->detmap) for (int d = 0; d < p->n_detmap; ++d) free(p->detmap[d]);
  if (p->obsmap) for (int d = 0; d < p->n_obsmap; ++d) free(p->obsmap[d]);
  free(p->detmap); free(p->detmap_n); free(p->obsmap); free(p->obsmap_n);
  free(p);
}

int oracle_info(const struct oracle_prog* p, int64_t* out) {
  out[0] = p->mode; out[1] = p->nx; out[2] = p->W; out[3] = p->nf; out[4] = p->nr;
  out[5] = p->nmeas; out[6] = p->ndet; out[7] = p->nobs; out[8] = p->n_out;
  out[9] = p->n_chains; out[10] = p->n_ch; out[11] = p->n_tab;
  out[12] = p->noise_mode; out[13] = p->n_groups;
  return 0;
}

/* outcome of a channel for the uniform word U: the smallest o < n-1 with
 * U < thr[o], else n-1 */
static int channel_outcome(const channel* ch, uint32_t U) {
  for (int j = 0; j + 1 < ch->n_out; ++j)
    if (U < ch->thr[j]) return j;
  return ch->n_out - 1;
}

/* Geometric gap: the number of non-candidates before the next candidate
 * among the m channels left in a group, i.e. the largest k <= m with
 * U < T_k (T_0 = 2^32 always holds), T_k given for k = 1..m. */
static int geo_gap(const uint32_t* T, int m, uint32_t U) {
  int k = 0;
  while (k < m && U < T[k + 1]) ++k;
  return k;
}

/* a word V mapped onto [Q, 2^32): Q + floor(V (2^32 - Q) / 2^32) */
static uint32_t geo_map(uint32_t Q, uint32_t V) {
  uint64_t R = ((uint64_t)1 << 32) - Q;
  return Q + (uint32_t)(((uint64_t)V * R) >> 32);
}

/* Exported for the pins: the gap for a group of m channels with the given Q
 * (the table built as the reader builds it), and the outcome of a candidate
 * channel with thresholds thr[0..n_out-2] for the word V. */
int oracle_geo_gap(uint32_t Q, int m, uint32_t U) {
  if (m < 0 || m > 1000000) return fail("bad group size");
  uint32_t* T = calloc((size_t)m + 1, sizeof(uint32_t));
  uint64_t t = (uint64_t)1 << 32;
  for (int k = 1; k <= m; ++k) {
    t = (t * (uint64_t)Q) >> 32;
    T[k] = (uint32_t)t;
  }
  int g = geo_gap(T, m, U);
  free(T);
  return g;
}

int oracle_geo_pick(uint32_t Q, const uint32_t* thr, int n_out, uint32_t V) {
  channel ch = {n_out, (uint32_t*)thr, NULL};
  if (n_out < 2 || thr[0] < Q) return fail("Q above the outcome-0 threshold");
  return channel_outcome(&ch, geo_map(Q, V));
}

/* parity of (mask & X) over W words: XOR of all selected bits, bit by bit */
static int parity(const uint64_t* mask, const uint64_t* X, int W) {
  int par = 0;
  for (int w = 0; w < W; ++w)
    for (int b = 0; b < 64; ++b)
      if ((mask[w] >> b) & 1) par ^= (int)((X[w] >> b) & 1);
  return par;
}

/* One factor of Table "Types of parameterized phase terms", from its formula
 * (angles in units of pi/4, w = e^{i pi/4}):
 *   kind 0 phase-pair  h = 1 + w^(alpha+4a) + w^(beta+4b) - w^(alpha+beta+4a+4b)
 *   kind 1 node        1 + w^(alpha+4a)
 *   kind 2 phase       w^(alpha*a)      (half-pi: alpha = +-2; sign: alpha = 4)
 *   kind 3 pi-pair     (-1)^(a b) = w^(4ab)                                      */
static int factor_value(const factor* fc, int a, int b, zw* out) {
  zw one = zw_omega(0);
  switch (fc->kind) {
    case 0: {
      zw x = zw_omega(fc->alpha + 4 * a), y = zw_omega(fc->beta + 4 * b);
      zw xy = zw_omega(fc->alpha + fc->beta + 4 * a + 4 * b);
      for (int i = 0; i < 4; ++i) xy.c[i] = -xy.c[i];
      *out = zw_add(zw_add(one, x), zw_add(y, xy));
      return 0;
    }
    case 1: *out = zw_add(one, zw_omega(fc->alpha + 4 * a)); return 0;
    case 2: *out = zw_omega(fc->alpha * a); return 0;
    case 3: *out = zw_omega(4 * a * b); return 0;
    default: return fail("unknown factor kind");
  }
}

/* P(X) = sum_t c^t prod_k h_k  with c^t = w^j0 sqrt2^s0 */
static int eval_table(const struct oracle_prog* p, int ti, const uint64_t* X, zw* out) {
  if (ti < 0 || ti >= p->n_tab) return fail("bad table index");
  const table* tb = &p->tab[ti];
  zw sum = zw_zero();
  for (int t = 0; t < tb->nt; ++t) {
    const term* tm = &tb->t[t];
    zw v = zw_omega(tm->j0);
    v.k = tm->s0;
    for (int k = 0; k < tm->nf; ++k) {
      const factor* fc = &tm->f[k];
      int a = parity(fc->u, X, p->W), b = parity(fc->v, X, p->W);
      zw h;
      if (factor_value(fc, a, b, &h)) return -1;
      v = zw_mul(v, h);
      if (zw_is_zero(&v)) break;
    }
    if (!zw_is_zero(&v)) sum = zw_add(sum, v);
  }
  *out = sum;
  return 0;
}

/* ---------------------------------------------------- floating-point tables */
typedef struct { double re, im; } cplx;

static cplx c_mul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }

/* an exact value (c0 + c1 w + c2 w^2 + c3 w^3) sqrt2^k in complex double */
static cplx zw_complex(const zw* z) {
  const double h = sqrt(0.5);
  cplx r = {(double)z->c[0] + h * ((double)z->c[1] - (double)z->c[3]),
            (double)z->c[2] + h * ((double)z->c[1] + (double)z->c[3])};
  const double m = pow(sqrt(2.0), z->k);
  r.re *= m;
  r.im *= m;
  return r;
}

static cplx e_i_pi(double t) { cplx r = {cos(M_PI * t), sin(M_PI * t)}; return r; }

/* P(X) = sum_t c^t e^(i pi phase_t) prod_k h_k, every factor from its formula
 * (the exact kinds as elements of Z[w], then converted), in table order */
static int eval_table_c(const struct oracle_prog* p, int ti, const uint64_t* X, cplx* out) {
  if (ti < 0 || ti >= p->n_tab) return fail("bad table index");
  const table* tb = &p->tab[ti];
  cplx sum = {0, 0};
  for (int t = 0; t < tb->nt; ++t) {
    const term* tm = &tb->t[t];
    zw c = zw_omega(tm->j0);
    c.k = tm->s0;
    cplx v = c_mul(zw_complex(&c), e_i_pi(tm->fph));
    for (int k = 0; k < tm->nf; ++k) {
      const factor* fc = &tm->f[k];
      int a = parity(fc->u, X, p->W), b = parity(fc->v, X, p->W);
      cplx h;
      if (fc->kind == 4) {
        h = a ? e_i_pi(fc->t) : (cplx){1.0, 0.0};
      } else {
        zw hz;
        if (factor_value(fc, a, b, &hz)) return -1;
        h = zw_complex(&hz);
      }
      v = c_mul(v, h);
    }
    sum.re += v.re;
    sum.im += v.im;
  }
  *out = sum;
  return 0;
}

/* Exported for the parity tests: the value of any table in complex double. */
int oracle_eval_table_c(const struct oracle_prog* p, int ti, const uint64_t* X, double* re_im) {
  g_ovf = 0;
  cplx z;
  if (eval_table_c(p, ti, X, &z)) return -1;
  if (g_ovf) return fail("int128 overflow in table evaluation");
  re_im[0] = z.re;
  re_im[1] = z.im;
  return 0;
}

/* Exported for the parity tests: value of one table at X, as
 * c[0..3] (each as hi,lo int64 pairs) and the sqrt2 exponent. */
int oracle_eval_table(const struct oracle_prog* p, int ti, const uint64_t* X, int64_t* coef8, int* k) {
  g_ovf = 0;
  if (ti >= 0 && ti < p->n_tab && p->tab[ti].flt) return fail("table has arbitrary phases");
  zw z;
  if (eval_table(p, ti, X, &z)) return -1;
  if (g_ovf) return fail("int128 overflow in table evaluation");
  for (int i = 0; i < 4; ++i) {
    coef8[2 * i] = (int64_t)(z.c[i] >> 64);
    coef8[2 * i + 1] = (int64_t)(uint64_t)z.c[i];
  }
  *k = z.k;
  return 0;
}

/* the j in 0..7 for which w^-j z is real and positive */
static int chain_phase(const zw* z, int* rot) {
  for (int j = 0; j < 8; ++j) {
    zw r = zw_mul(*z, zw_omega(-j));
    if (r.c[2] == 0 && add_(r.c[1], r.c[3]) == 0) {
      rv v;
      if (zw_to_real(&r, &v)) return -1;
      if (sign_xy(v.A, v.B) > 0) { *rot = j; return 0; }
    }
  }
  return fail("normalisation has no positive real phase");
}

/* 1-2: error mechanisms and f = T e, into X (W words, zeroed first) */
static void sample_noise(const struct oracle_prog* p, uint64_t seed, uint64_t shot, uint64_t* X) {
  int W = p->W;
  memset(X, 0, (size_t)W * 8);
  if (p->noise_mode == 0) {
    for (int c = 0; c < p->n_ch; ++c) {
      const channel* ch = &p->ch[c];
      uint32_t U = philox_word(seed, shot, 0, (uint32_t)c);
      int o = channel_outcome(ch, U);
      for (int w = 0; w < W; ++w) X[w] ^= ch->sig[(size_t)o * W + w];
    }
  } else {
    uint32_t j = 0;  /* next word of stream 2 */
    for (int g = 0; g < p->n_groups; ++g) {
      const group* G = &p->groups[g];
      int pos = 0;
      while (pos < G->n) {
        uint32_t U = philox_word(seed, shot, 2, j++);
        pos += geo_gap(G->T, G->n - pos, U);
        if (pos >= G->n) break;
        const channel* ch = &p->ch[G->member[pos]];
        uint32_t V = philox_word(seed, shot, 2, j++);
        int o = channel_outcome(ch, geo_map(G->Q, V));
        for (int w = 0; w < W; ++w) X[w] ^= ch->sig[(size_t)o * W + w];
        pos += 1;
      }
    }
  }
}

/* Exported for the parity tests: X = T e of one shot, before any output. */
int oracle_noise_x(const struct oracle_prog* p, uint64_t seed, uint64_t shot, uint64_t* X) {
  sample_noise(p, seed, shot, X);
  return 0;
}

static int sample_shot(const struct oracle_prog* p, uint64_t seed, uint64_t shot, uint64_t* X,
                       uint8_t* bits, rv* pprev, int* rot, double* fprev, cplx* fnorm) {
  int W = p->W;
  sample_noise(p, seed, shot, X);
  /* Algorithm 1: P_prev <- P for every chain (phase removed) */
  for (int c = 0; c < p->n_chains; ++c) {
    if (p->chain_float[c]) {
      cplx z;
      if (eval_table_c(p, p->chain_norm[c], X, &z)) return -1;
      const double m = sqrt(z.re * z.re + z.im * z.im);
      if (!(m > 0)) return fail("normalisation is zero");
      fnorm[c] = z;
      fprev[c] = m;
      continue;
    }
    zw z;
    if (eval_table(p, p->chain_norm[c], X, &z)) return -1;
    if (chain_phase(&z, &rot[c])) return -1;
    z = zw_mul(z, zw_omega(-rot[c]));
    if (zw_to_real(&z, &pprev[c])) return -1;
  }
  /* 3: outputs in autoregressive order */
  for (int i = 0; i < p->n_out; ++i) {
    const output* o = &p->out[i];
    int bit;
    if (!o->is_random) {
      bit = parity(o->mask, X, W) ^ o->cst;
    } else {
      int xb = o->xbit;
      X[xb >> 6] |= (uint64_t)1 << (xb & 63);
      if (p->chain_float[o->chain]) {
        const int c = o->chain;
        cplx z1;
        if (eval_table_c(p, o->table, X, &z1)) return -1;
        const cplx zn = fnorm[c];
        const double mn = sqrt(zn.re * zn.re + zn.im * zn.im);
        const double p1 = (z1.re * zn.re + z1.im * zn.im) / mn;
        if (!(fprev[c] > 0)) return fail("P_prev is not positive");
        const float q = (float)(p1 / fprev[c]);
        uint32_t U = philox_word(seed, shot, 1, (uint32_t)i);
        bit = (double)U < (double)q * 4294967296.0;
        if (bit) {
          fprev[c] = p1;
        } else {
          fprev[c] = fprev[c] - p1;
          X[xb >> 6] &= ~((uint64_t)1 << (xb & 63));
        }
        bits[i] = (uint8_t)bit;
        continue;
      }
      zw z;
      rv p1;
      if (eval_table(p, o->table, X, &z)) return -1;
      z = zw_mul(z, zw_omega(-rot[o->chain]));
      if (zw_to_real(&z, &p1)) return -1;
      rv pp = pprev[o->chain];
      if (sign_xy(pp.A, pp.B) <= 0) return fail("P_prev is not positive");
      uint32_t U = philox_word(seed, shot, 1, (uint32_t)i);
      /* bit = 1 iff U * P_prev < 2^32 * P_1 */
      rv lhs = {mul_(pp.A, (i128)U), mul_(pp.B, (i128)U), pp.e};
      rv rhs = {p1.A, p1.B, p1.e + 32};
      rv_align(&lhs, &rhs);
      bit = sign_xy(sub_(lhs.A, rhs.A), sub_(lhs.B, rhs.B)) < 0;
      if (bit) {
        pprev[o->chain] = p1;
      } else {
        rv a = pp, b = p1;
        rv_align(&a, &b);
        rv d = {sub_(a.A, b.A), sub_(a.B, b.B), a.e};
        pprev[o->chain] = d;
        X[xb >> 6] &= ~((uint64_t)1 << (xb & 63));
      }
    }
    bits[i] = (uint8_t)bit;
  }
  return 0;
}

/* Sample shots [shot_begin, shot_begin + n) into bit-packed rows:
 * meas[n][ceil(nmeas/64)] (measurement mode), det[n][ceil(ndet/64)],
 * obs[n][ceil(nobs/64)], accept[n].  Any pointer may be NULL. */
int oracle_sample(const struct oracle_prog* p, uint64_t seed, uint64_t shot_begin, uint64_t n,
                  uint64_t* meas, uint64_t* det, uint64_t* obs, uint8_t* accept) {
  g_ovf = 0;
  int W = p->W;
  int wm = (p->nmeas + 63) / 64, wd = (p->ndet + 63) / 64, wo = (p->nobs + 63) / 64;
  uint64_t* X = calloc((size_t)W, 8);
  uint8_t* bits = calloc((size_t)p->n_out + 1, 1);
  rv* pprev = calloc((size_t)p->n_chains + 1, sizeof(rv));
  int* rot = calloc((size_t)p->n_chains + 1, sizeof(int));
  double* fprev = calloc((size_t)p->n_chains + 1, sizeof(double));
  cplx* fnorm = calloc((size_t)p->n_chains + 1, sizeof(cplx));
  int rc = 0;
  for (uint64_t s = 0; s < n; ++s) {
    if (sample_shot(p, seed, shot_begin + s, X, bits, pprev, rot, fprev, fnorm)) { rc = -1; break; }
    if (g_ovf) { rc = fail("int128 overflow while sampling"); break; }
    uint8_t dbits[4096];
    int nd = p->ndet;
    if (nd > 4096) { rc = fail("too many detectors for the oracle"); break; }
    if (p->mode == 0) {
      for (int d = 0; d < nd; ++d) dbits[d] = bits[d];
    } else {
      for (int d = 0; d < nd; ++d) {
        int v = 0;
        for (int j = 0; j < p->detmap_n[d]; ++j) v ^= bits[p->detmap[d][j]];
        dbits[d] = (uint8_t)v;
      }
    }
    if (meas && p->mode == 1) {
      uint64_t* row = meas + s * wm;
      memset(row, 0, (size_t)wm * 8);
      for (int m = 0; m < p->nmeas; ++m) row[m >> 6] |= (uint64_t)bits[m] << (m & 63);
    }
    if (det) {
      uint64_t* row = det + s * wd;
      memset(row, 0, (size_t)wd * 8);
      for (int d = 0; d < nd; ++d) row[d >> 6] |= (uint64_t)dbits[d] << (d & 63);
    }
    if (obs) {
      uint64_t* row = obs + s * wo;
      memset(row, 0, (size_t)wo * 8);
      for (int k = 0; k < p->nobs; ++k) {
        int v;
        if (p->mode == 0) v = bits[nd + k];
        else {
          v = 0;
          for (int j = 0; j < p->obsmap_n[k]; ++j) v ^= bits[p->obsmap[k][j]];
        }
        row[k >> 6] |= (uint64_t)v << (k & 63);
      }
    }
    if (accept) {
      int ok = 1;
      for (int d = 0; d < nd; ++d) if (dbits[d]) { ok = 0; break; }
      accept[s] = (uint8_t)ok;
    }
  }
  free(X); free(bits); free(pprev); free(rot); free(fprev); free(fnorm);
  return rc;
}

/* Exact Bernoulli decision exported for pins: bit for a uniform word U and
 * probabilities given as (A + B sqrt2) * 2^e. */
int oracle_decide(uint32_t U, int64_t Ap, int64_t Bp, int ep, int64_t A1, int64_t B1, int e1) {
  g_ovf = 0;
  rv lhs = {mul_((i128)Ap, (i128)U), mul_((i128)Bp, (i128)U), ep};
  rv rhs = {(i128)A1, (i128)B1, e1 + 32};
  rv_align(&lhs, &rhs);
  int bit = sign_xy(sub_(lhs.A, rhs.A), sub_(lhs.B, rhs.B)) < 0;
  if (g_ovf) return fail("overflow");
  return bit;
}
