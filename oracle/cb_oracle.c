/*
 * ORACLE (test infrastructure).  A plain, slow, sequential CPU statement of
 * the undirected global Curveball super step.  Only tests/, the smoke check in
 * __graft_entry__ and bench.py's cpu_baseline / reference leg may load it; the
 * CUDA library shares no code, header, table or helper with it.
 *
 * What it computes, in the paper's order and notation:
 *
 *  - Def. "Undirected Global Trade" (Section 3.3): a permutation pi of the
 *    nodes pairs positions (2i-1, 2i) into l = floor(n/2) trades
 *    t_i = {pi(v_{2i-1}), pi(v_{2i})}, applied successively in index order.
 *    For odd n the node at the last position is not traded (Section 1
 *    footnote; Section 3.3 "add an isolated node").
 *  - Def. "Simple Undirected Trade" (Section 3.2) and Fig. 2: for a trade of
 *    i and j, A_{i-j} = A_i \ (A_j u {j}), D = A_{i-j} u A_{j-i}; a
 *    permutation sigma of D is drawn and i receives the first |A_{i-j}|
 *    elements of sigma(D), j the rest (Fig. 2 fixes the rank convention);
 *    symmetry is kept by relabelling the passive neighbours.
 *  - Section 4 (trading procedure): sigma is chosen by the algorithm for each
 *    trade, uniformly; |A_u n D| elements of D go to u.
 *
 * Readings where the paper leaves the choice open:
 *  - pi: node x gets the 64-bit key philox64(seed; x, 0, g, 0) (counter
 *    words c0..c3), nodes are sorted by (key, id), 0-based positions, and
 *    trade t (0-based) is (order[2t], order[2t+1]).
 *  - sigma: every edge present at the start of super step g is identified by
 *    the positions (lo < hi) of its two endpoints at that time.  Philox4x32-10
 *    on counter (lo, hi, g, 1) gives four words r0..r3; the trade owning
 *    position lo keys the edge with (r0<<32|r1), the trade owning position hi
 *    with (r2<<32|r3).  A disjoint neighbour x of trade t is keyed by the edge
 *    joining x to {u_t, v_t}; sigma(D) is D sorted by (key, lo, hi).
 *  - Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
 *    Easy as 1, 2, 3" (SC'11); key words (k0, k1) = (low, high) 32 bits of the
 *    seed; philox64 = (r0 << 32) | r1.
 *  - Uniform single trades (Simple Undirected Curveball, Section 3.2, the
 *    paragraph after Fig. 2; the trade sequence T of Section 4.1): trade i
 *    (0-based, 64-bit) draws Philox4x32-10 on counter (i_lo, i_hi, 0, 5) =
 *    r0..r3; u = floor(r0 n / 2^32), w = floor(r1 (n-1) / 2^32) and
 *    v = w + (w >= u), so u != v and every ordered pair has probability
 *    1/(n(n-1)) up to a relative 2^-32.  sigma: disjoint neighbour x (node
 *    id) is keyed by (r0<<32|r1) of Philox4x32-10 on counter
 *    (x, i_lo, i_hi, 6); sigma(D) is D sorted by (key, x).  The trades apply
 *    one after the other in index order.
 *  - Swap counts (Appendix "Swaps performed by Curveball and Global
 *    Curveball"): a trade performs as many neighbourhood swaps as edge ends
 *    that change node (twice the pairs of neighbours exchanged; Fig. 2's
 *    sigma exchanges four edges), out of deg(u) + deg(v) possible.
 *  - Relaxed global trade (Def. "Relaxed global trade", Appendix EM-GCB; the
 *    linear congruential maps of Section 4.3 and the Appendix "Linear
 *    congruential maps"), when switched on: super step g draws
 *    h(x) = (a x + b) mod p, p the smallest prime >= n, from Philox4x32-10 on
 *    counter (0, 0, g, 4) = r0..r3: a = 1 + ((r0<<32|r1) mod (p-1)),
 *    b = (r2<<32|r3) mod p.  The nodes in order of h(x) (injective on [n])
 *    form the trades, as a permutation does.
 *
 * Data structure: the edge list E (two endpoint fields per edge, plus the
 * edge's identity at the start of the current super step) and, per node, the
 * list of incident edge ids.  A trade rewrites the endpoint field of each edge
 * it moves and exchanges the moved edge ids between the lists of its two
 * nodes; the passive neighbour's own list is untouched because it stores edge
 * ids, not node ids.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ERANGE (-3)

/* ------------------------------------------------------------------ Philox */
static void philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Exported for the pin against an independent Philox implementation. */
void or_philox4x32_10(const uint32_t* ctr, uint64_t seed, uint32_t* out) {
  philox4x32_10(ctr, seed, out);
}

/* ------------------------------------------------------------------- state */
typedef struct {
  int64_t n, m;
  uint64_t seed, g;        /* g = index of the next super step */
  int64_t* row_ptr;        /* incidence-list offsets (degrees never change) */
  uint32_t* inc;           /* incident edge ids per node */
  int32_t* end;            /* end[2e], end[2e+1]: current endpoints of edge e */
  uint32_t* id_lo;         /* identity of edge e at the start of the step */
  uint32_t* id_hi;
  int64_t* pos;            /* position of each node in the current step */
  int64_t* order;          /* node at each position */
  int64_t maxdeg;
  int relaxed;             /* 1: permutations from linear congruential maps */
  uint64_t uni;            /* index of the next uniform single trade */
  int64_t swaps_done;      /* edge ends that changed node in a trade (2 per exchanged pair) */
  int64_t swaps_all;       /* deg(u) + deg(v) summed over the trades */
  /* per-trade scratch */
  void* scratch;
} or_state;

typedef struct { int32_t other; uint32_t e; int64_t slot; } nbr;            /* one incident edge */
typedef struct { int32_t x; uint32_t e; int64_t slot; int side; uint64_t key; uint32_t lo, hi; } elem;
typedef struct { uint64_t key; int64_t id; } keyid;

static int cmp_nbr(const void* p, const void* q) {
  const nbr* a = (const nbr*)p; const nbr* b = (const nbr*)q;
  return (a->other > b->other) - (a->other < b->other);
}
static int cmp_keyid(const void* p, const void* q) {
  const keyid* a = (const keyid*)p; const keyid* b = (const keyid*)q;
  if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
  return (a->id > b->id) - (a->id < b->id);
}
static int cmp_sigma(const void* p, const void* q) {
  const elem* a = (const elem*)p; const elem* b = (const elem*)q;
  if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
  if (a->lo != b->lo) return (a->lo > b->lo) - (a->lo < b->lo);
  return (a->hi > b->hi) - (a->hi < b->hi);
}
static int cmp_i32(const void* p, const void* q) {
  int32_t a = *(const int32_t*)p, b = *(const int32_t*)q;
  return (a > b) - (a < b);
}
static int cmp_u64(const void* p, const void* q) {
  uint64_t a = *(const uint64_t*)p, b = *(const uint64_t*)q;
  return (a > b) - (a < b);
}

typedef struct { nbr* au; nbr* av; elem* d; } scratch_t;

void or_destroy(void* hp) {
  or_state* h = (or_state*)hp;
  if (!h) return;
  free(h->row_ptr); free(h->inc); free(h->end); free(h->id_lo); free(h->id_hi);
  free(h->pos); free(h->order);
  if (h->scratch) {
    scratch_t* s = (scratch_t*)h->scratch;
    free(s->au); free(s->av); free(s->d); free(s);
  }
  free(h);
}

/*
 * Build the oracle state from a CSR adjacency (row_ptr: n+1 entries, col:
 * row_ptr[n] entries).  The graph must be simple and symmetric.  Returns NULL
 * with *rc set on error.
 */
void* or_create(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed,
                uint64_t first_step, int* rc) {
  *rc = OR_EINVAL;
  if (n < 0 || n > 0x7fffffffLL || !row_ptr || (row_ptr[n] > 0 && !col)) return NULL;
  if (first_step > 0xffffffffULL) { *rc = OR_ERANGE; return NULL; }
  int64_t nnz = row_ptr[n];
  if (row_ptr[0] != 0 || (nnz & 1)) return NULL;
  for (int64_t x = 0; x < n; x++) if (row_ptr[x + 1] < row_ptr[x]) return NULL;
  if (nnz / 2 > 0xffffffffLL) { *rc = OR_ERANGE; return NULL; }
  /* simple + symmetric: check on row-sorted copies */
  int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
  if (!sc) { *rc = OR_ENOMEM; return NULL; }
  memcpy(sc, col, sizeof(int32_t) * (size_t)nnz);
  for (int64_t x = 0; x < n; x++)
    qsort(sc + row_ptr[x], (size_t)(row_ptr[x + 1] - row_ptr[x]), sizeof(int32_t), cmp_i32);
  for (int64_t x = 0; x < n; x++) {
    for (int64_t q = row_ptr[x]; q < row_ptr[x + 1]; q++) {
      int32_t y = sc[q];
      if (y < 0 || y >= n || y == x || (q > row_ptr[x] && sc[q - 1] == y)) { free(sc); return NULL; }
      /* y must list x */
      int64_t lo = row_ptr[y], hi = row_ptr[y + 1];
      while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (sc[mid] < x) lo = mid + 1; else hi = mid; }
      if (lo == row_ptr[y + 1] || sc[lo] != x) { free(sc); return NULL; }
    }
  }
  or_state* h = (or_state*)calloc(1, sizeof(or_state));
  if (!h) { free(sc); *rc = OR_ENOMEM; return NULL; }
  h->n = n; h->m = nnz / 2; h->seed = seed; h->g = first_step;
  h->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  h->inc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nnz ? nnz : 1));
  h->end = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * h->m + 2));
  h->id_lo = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(h->m + 1));
  h->id_hi = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(h->m + 1));
  h->pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  h->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  scratch_t* s = (scratch_t*)calloc(1, sizeof(scratch_t));
  h->scratch = s;
  int64_t maxdeg = 0;
  for (int64_t x = 0; x < n; x++) if (row_ptr[x + 1] - row_ptr[x] > maxdeg) maxdeg = row_ptr[x + 1] - row_ptr[x];
  h->maxdeg = maxdeg;
  if (s) {
    s->au = (nbr*)malloc(sizeof(nbr) * (size_t)(maxdeg + 1));
    s->av = (nbr*)malloc(sizeof(nbr) * (size_t)(maxdeg + 1));
    s->d = (elem*)malloc(sizeof(elem) * (size_t)(2 * maxdeg + 1));
  }
  if (!h->row_ptr || !h->inc || !h->end || !h->id_lo || !h->id_hi || !h->pos || !h->order || !s ||
      !s->au || !s->av || !s->d) {
    free(sc); or_destroy(h); *rc = OR_ENOMEM; return NULL;
  }
  memcpy(h->row_ptr, row_ptr, sizeof(int64_t) * (size_t)(n + 1));
  /* edge ids in canonical order: edge [x,y], x<y, numbered by (x, y) */
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!fill) { free(sc); or_destroy(h); *rc = OR_ENOMEM; return NULL; }
  for (int64_t x = 0; x < n; x++) fill[x] = row_ptr[x];
  uint32_t e = 0;
  for (int64_t x = 0; x < n; x++) {
    for (int64_t q = row_ptr[x]; q < row_ptr[x + 1]; q++) {
      int32_t y = sc[q];
      if (y > x) {
        h->end[2 * (int64_t)e] = (int32_t)x; h->end[2 * (int64_t)e + 1] = y;
        h->inc[fill[x]++] = e; h->inc[fill[y]++] = e;
        e++;
      }
    }
  }
  free(fill); free(sc);
  *rc = OR_OK;
  return h;
}

uint64_t or_step(void* hp) { return ((or_state*)hp)->g; }
int64_t or_num_edges(void* hp) { return ((or_state*)hp)->m; }
int64_t or_num_nodes(void* hp) { return ((or_state*)hp)->n; }

/* Smallest prime p >= n (trial division; p = 2 for n <= 2). */
static uint64_t next_prime(uint64_t n) {
  for (uint64_t p = n < 2 ? 2 : n;; p++) {
    int prime = 1;
    for (uint64_t d = 2; d * d <= p; d++)
      if (p % d == 0) { prime = 0; break; }
    if (prime) return p;
  }
}

/* The linear congruential map h(x) = (a x + b) mod p of super step g. */
static void lcg_params(const or_state* h, uint64_t g, uint64_t* p, uint64_t* a, uint64_t* b) {
  uint32_t ctr[4] = {0u, 0u, (uint32_t)g, 4u}, r[4];
  philox4x32_10(ctr, h->seed, r);
  *p = next_prime((uint64_t)h->n);
  *a = 1 + ((((uint64_t)r[0] << 32) | r[1]) % (*p - 1));
  *b = (((uint64_t)r[2] << 32) | r[3]) % *p;
}

void or_lcg_params(void* hp, uint64_t g, uint64_t* p, uint64_t* a, uint64_t* b) {
  lcg_params((or_state*)hp, g, p, a, b);
}

void or_set_relaxed(void* hp, int on) { ((or_state*)hp)->relaxed = on != 0; }

/* Permutation pi for super step g: positions of all nodes. */
static int compute_permutation(or_state* h, uint64_t g) {
  keyid* ki = (keyid*)malloc(sizeof(keyid) * (size_t)(h->n ? h->n : 1));
  if (!ki) return OR_ENOMEM;
  uint64_t p = 0, a = 0, b = 0;
  if (h->relaxed) lcg_params(h, g, &p, &a, &b);
  for (int64_t x = 0; x < h->n; x++) {
    if (h->relaxed) {
      ki[x].key = (a * (uint64_t)x + b) % p;   /* the image h(x): distinct for x < n <= p */
    } else {
      uint32_t ctr[4] = {(uint32_t)x, 0u, (uint32_t)g, 0u}, r[4];
      philox4x32_10(ctr, h->seed, r);
      ki[x].key = ((uint64_t)r[0] << 32) | r[1];
    }
    ki[x].id = x;
  }
  qsort(ki, (size_t)h->n, sizeof(keyid), cmp_keyid);
  for (int64_t p = 0; p < h->n; p++) { h->order[p] = ki[p].id; h->pos[ki[p].id] = p; }
  free(ki);
  return OR_OK;
}

/* Positions of the super step about to run (for tests of the permutation). */
int or_permutation(void* hp, uint64_t g, int64_t* order_out) {
  or_state* h = (or_state*)hp;
  if (g > 0xffffffffULL) return OR_ERANGE;
  int rc = compute_permutation(h, g);
  if (rc) return rc;
  memcpy(order_out, h->order, sizeof(int64_t) * (size_t)h->n);
  return OR_OK;
}

/*
 * Gather the current neighbourhoods of u and v and split them into the
 * disjoint set D (Def. "Simple Undirected Trade"): elements adjacent to
 * exactly one of u, v, excluding u and v themselves.  Returns |D| and sets
 * *a = |A_{u-v}|.  Elements come out ordered by node id.
 */
static int64_t disjoint_set(or_state* h, int64_t u, int64_t v, elem* d, int64_t* a) {
  scratch_t* s = (scratch_t*)h->scratch;
  int64_t du = h->row_ptr[u + 1] - h->row_ptr[u], dv = h->row_ptr[v + 1] - h->row_ptr[v];
  for (int64_t i = 0; i < du; i++) {
    int64_t slot = h->row_ptr[u] + i; uint32_t e = h->inc[slot];
    int32_t o = h->end[2 * (int64_t)e] == u ? h->end[2 * (int64_t)e + 1] : h->end[2 * (int64_t)e];
    s->au[i].other = o; s->au[i].e = e; s->au[i].slot = slot;
  }
  for (int64_t i = 0; i < dv; i++) {
    int64_t slot = h->row_ptr[v] + i; uint32_t e = h->inc[slot];
    int32_t o = h->end[2 * (int64_t)e] == v ? h->end[2 * (int64_t)e + 1] : h->end[2 * (int64_t)e];
    s->av[i].other = o; s->av[i].e = e; s->av[i].slot = slot;
  }
  qsort(s->au, (size_t)du, sizeof(nbr), cmp_nbr);
  qsort(s->av, (size_t)dv, sizeof(nbr), cmp_nbr);
  int64_t i = 0, j = 0, k = 0, na = 0;
  while (i < du || j < dv) {
    if (j >= dv || (i < du && s->au[i].other < s->av[j].other)) {        /* only in A_u */
      if (s->au[i].other != v) {
        d[k].x = s->au[i].other; d[k].e = s->au[i].e; d[k].slot = s->au[i].slot; d[k].side = 0; k++; na++;
      }
      i++;
    } else if (i >= du || s->av[j].other < s->au[i].other) {             /* only in A_v */
      if (s->av[j].other != u) {
        d[k].x = s->av[j].other; d[k].e = s->av[j].e; d[k].slot = s->av[j].slot; d[k].side = 1; k++;
      }
      j++;
    } else { i++; j++; }                                                  /* common: kept */
  }
  *a = na;
  return k;
}

/*
 * Apply a trade of u and v given sigma(D) as a sequence of elements: u gets
 * the first a of them, v the rest (Fig. 2).  Each element whose side changes
 * has its edge moved: the endpoint field naming the old node is rewritten and
 * the edge id moves to the other node's incidence list.  Moves come in pairs
 * (as many leave u as arrive), so each pair exchanges incidence-list slots.
 */
static void apply_sigma(or_state* h, int64_t u, int64_t v, elem* sig, int64_t nd, int64_t a) {
  /* walk the u->v movers and v->u movers in sigma order and pair them */
  int64_t p = 0, q = 0;
  for (;;) {
    while (p < nd && !(sig[p].side == 0 && p >= a)) p++;   /* was at u, goes to v */
    while (q < nd && !(sig[q].side == 1 && q < a)) q++;    /* was at v, goes to u */
    if (p >= nd || q >= nd) break;
    elem* x = &sig[p]; elem* y = &sig[q];
    /* edge x->e: endpoint u becomes v; edge y->e: endpoint v becomes u */
    if (h->end[2 * (int64_t)x->e] == u) h->end[2 * (int64_t)x->e] = (int32_t)v; else h->end[2 * (int64_t)x->e + 1] = (int32_t)v;
    if (h->end[2 * (int64_t)y->e] == v) h->end[2 * (int64_t)y->e] = (int32_t)u; else h->end[2 * (int64_t)y->e + 1] = (int32_t)u;
    h->inc[x->slot] = y->e;   /* slot in u's list now holds the edge arriving at u */
    h->inc[y->slot] = x->e;   /* slot in v's list now holds the edge arriving at v */
    h->swaps_done += 2;
    p++; q++;
  }
  h->swaps_all += (h->row_ptr[u + 1] - h->row_ptr[u]) + (h->row_ptr[v + 1] - h->row_ptr[v]);
}

/* One trade of the global trade: sigma drawn from the edge keys of step g. */
static void trade(or_state* h, int64_t t, uint64_t g) {
  scratch_t* s = (scratch_t*)h->scratch;
  int64_t u = h->order[2 * t], v = h->order[2 * t + 1], a;
  int64_t nd = disjoint_set(h, u, v, s->d, &a);
  for (int64_t k = 0; k < nd; k++) {
    uint32_t e = s->d[k].e, lo = h->id_lo[e], hi = h->id_hi[e], r[4];
    uint32_t ctr[4] = {lo, hi, (uint32_t)g, 1u};
    philox4x32_10(ctr, h->seed, r);
    s->d[k].lo = lo; s->d[k].hi = hi;
    /* the edge's endpoint on trade t's side sat at position lo or hi */
    s->d[k].key = ((int64_t)(lo >> 1) == t) ? (((uint64_t)r[0] << 32) | r[1])
                                             : (((uint64_t)r[2] << 32) | r[3]);
  }
  qsort(s->d, (size_t)nd, sizeof(elem), cmp_sigma);   /* sigma(D) */
  apply_sigma(h, u, v, s->d, nd, a);
}

/* Run `count` super steps. */
int or_superstep(void* hp, uint32_t count) {
  or_state* h = (or_state*)hp;
  for (uint32_t c = 0; c < count; c++) {
    if (h->g > 0xffffffffULL) return OR_ERANGE;
    uint64_t g = h->g;
    int rc = compute_permutation(h, g);
    if (rc) return rc;
    for (int64_t e = 0; e < h->m; e++) {
      int64_t pa = h->pos[h->end[2 * e]], pb = h->pos[h->end[2 * e + 1]];
      h->id_lo[e] = (uint32_t)(pa < pb ? pa : pb);
      h->id_hi[e] = (uint32_t)(pa < pb ? pb : pa);
    }
    int64_t T = h->n / 2;
    for (int64_t t = 0; t < T; t++) trade(h, t, g);
    h->g = g + 1;
  }
  return OR_OK;
}

/*
 * Trade u and v with an explicitly given sigma(D) (node ids, a permutation of
 * the current disjoint set D).  Used to check the trade primitive against the
 * worked example of Fig. 2.  Returns OR_EINVAL if sigma is not a permutation
 * of D.
 */
int or_trade_explicit(void* hp, int64_t u, int64_t v, const int32_t* sigma, int64_t len) {
  or_state* h = (or_state*)hp;
  scratch_t* s = (scratch_t*)h->scratch;
  if (u < 0 || v < 0 || u >= h->n || v >= h->n || u == v) return OR_EINVAL;
  int64_t a, nd = disjoint_set(h, u, v, s->d, &a);
  if (len != nd) return OR_EINVAL;
  elem* tmp = (elem*)malloc(sizeof(elem) * (size_t)(nd ? nd : 1));
  if (!tmp) return OR_ENOMEM;
  for (int64_t k = 0; k < nd; k++) {
    int64_t lo = 0, hi = nd;                 /* D is ordered by node id */
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (s->d[mid].x < sigma[k]) lo = mid + 1; else hi = mid; }
    if (lo == nd || s->d[lo].x != sigma[k]) { free(tmp); return OR_EINVAL; }
    tmp[k] = s->d[lo];
  }
  for (int64_t k = 0; k < nd; k++)
    for (int64_t l = k + 1; l < nd; l++)
      if (tmp[k].x == tmp[l].x) { free(tmp); return OR_EINVAL; }
  apply_sigma(h, u, v, tmp, nd, a);
  free(tmp);
  return OR_OK;
}

/* Current disjoint set of u, v (node ids ascending); returns |D|, *a = |A_{u-v}|. */
int64_t or_disjoint(void* hp, int64_t u, int64_t v, int32_t* out, int64_t cap, int64_t* a) {
  or_state* h = (or_state*)hp;
  scratch_t* s = (scratch_t*)h->scratch;
  if (u < 0 || v < 0 || u >= h->n || v >= h->n || u == v) return OR_EINVAL;
  int64_t nd = disjoint_set(h, u, v, s->d, a);
  if (nd > cap) return OR_ERANGE;
  for (int64_t k = 0; k < nd; k++) out[k] = s->d[k].x;
  return nd;
}

/* ------------------------------------------------- uniform single trades */

/* The node pair of uniform trade i on n >= 2 nodes (see the header). */
void or_uniform_pair(uint64_t seed, int64_t n, uint64_t i, int64_t* u, int64_t* v) {
  uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0u, 5u}, r[4];
  philox4x32_10(ctr, seed, r);
  int64_t a = (int64_t)(((uint64_t)r[0] * (uint64_t)n) >> 32);
  int64_t w = (int64_t)(((uint64_t)r[1] * (uint64_t)(n - 1)) >> 32);
  *u = a;
  *v = w + (w >= a);
}

static int cmp_key_x(const void* p, const void* q) {
  const elem* a = (const elem*)p; const elem* b = (const elem*)q;
  if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
  return (a->x > b->x) - (a->x < b->x);
}

/* Uniform trade i: the drawn pair, D, sigma(D) by the keys of trade i, Fig. 2. */
static void uniform_trade(or_state* h, uint64_t i) {
  scratch_t* s = (scratch_t*)h->scratch;
  int64_t u, v, a;
  or_uniform_pair(h->seed, h->n, i, &u, &v);
  int64_t nd = disjoint_set(h, u, v, s->d, &a);
  for (int64_t k = 0; k < nd; k++) {
    uint32_t ctr[4] = {(uint32_t)s->d[k].x, (uint32_t)i, (uint32_t)(i >> 32), 6u}, r[4];
    philox4x32_10(ctr, h->seed, r);
    s->d[k].key = ((uint64_t)r[0] << 32) | r[1];
  }
  qsort(s->d, (size_t)nd, sizeof(elem), cmp_key_x);   /* sigma(D) */
  apply_sigma(h, u, v, s->d, nd, a);
}

/* Apply the next `count` uniform trades (none exist for n < 2: only the index advances). */
int or_uniform_trades(void* hp, uint64_t count) {
  or_state* h = (or_state*)hp;
  for (uint64_t c = 0; c < count; c++) {
    if (h->n >= 2) uniform_trade(h, h->uni);
    h->uni++;
  }
  return OR_OK;
}

uint64_t or_uniform_next(void* hp) { return ((or_state*)hp)->uni; }
void or_set_uniform_next(void* hp, uint64_t i) { ((or_state*)hp)->uni = i; }

/* Swap counts since creation or the last reset (see the header). */
void or_swap_counts(void* hp, int64_t* performed, int64_t* possible, int reset) {
  or_state* h = (or_state*)hp;
  *performed = h->swaps_done;
  *possible = h->swaps_all;
  if (reset) { h->swaps_done = 0; h->swaps_all = 0; }
}

/*
 * Successor lists of a trade sequence (Section 4.1): for each node x the
 * increasing indices i of the trades t_i = {pairs[2i], pairs[2i+1]} that
 * contain x, in suc[begin[x] .. begin[x+1]); the closing "infinity" of the
 * paper is the end of the range.  Returns OR_EINVAL for a node outside [0, n)
 * or a pair of equal nodes.
 */
int or_successors(int64_t n, const int32_t* pairs, int64_t count, int64_t* begin, int32_t* suc) {
  for (int64_t x = 0; x <= n; x++) begin[x] = 0;
  for (int64_t i = 0; i < count; i++) {
    int32_t a = pairs[2 * i], b = pairs[2 * i + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) return OR_EINVAL;
    begin[a + 1]++; begin[b + 1]++;
  }
  for (int64_t x = 0; x < n; x++) begin[x + 1] += begin[x];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  if (!fill) return OR_ENOMEM;
  for (int64_t x = 0; x < n; x++) fill[x] = begin[x];
  for (int64_t i = 0; i < count; i++) {   /* increasing i: each list comes out sorted */
    suc[fill[pairs[2 * i]]++] = (int32_t)i;
    suc[fill[pairs[2 * i + 1]]++] = (int32_t)i;
  }
  free(fill);
  return OR_OK;
}

/* Canonical edge list: pairs [a,b] with a<b, sorted lexicographically. */
int64_t or_export(void* hp, int32_t* pairs, int64_t cap_pairs) {
  or_state* h = (or_state*)hp;
  if (cap_pairs < h->m) return OR_ERANGE;
  uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(h->m ? h->m : 1));
  if (!w) return OR_ENOMEM;
  for (int64_t e = 0; e < h->m; e++) {
    uint32_t a = (uint32_t)h->end[2 * e], b = (uint32_t)h->end[2 * e + 1];
    if (a > b) { uint32_t t = a; a = b; b = t; }
    w[e] = ((uint64_t)a << 32) | b;
  }
  qsort(w, (size_t)h->m, sizeof(uint64_t), cmp_u64);
  for (int64_t e = 0; e < h->m; e++) { pairs[2 * e] = (int32_t)(w[e] >> 32); pairs[2 * e + 1] = (int32_t)(uint32_t)w[e]; }
  free(w);
  return h->m;
}

/* Deep copy (for exact enumeration in tests). */
void* or_clone(void* hp, int* rc) {
  or_state* h = (or_state*)hp;
  int64_t nnz = h->row_ptr[h->n];
  /* rebuild from the current adjacency */
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(h->n + 1));
  if (!col || !fill) { free(col); free(fill); *rc = OR_ENOMEM; return NULL; }
  for (int64_t x = 0; x < h->n; x++) fill[x] = h->row_ptr[x];
  for (int64_t e = 0; e < h->m; e++) {
    int32_t a = h->end[2 * e], b = h->end[2 * e + 1];
    col[fill[a]++] = b; col[fill[b]++] = a;
  }
  void* c = or_create(h->n, h->row_ptr, col, h->seed, h->g, rc);
  free(col); free(fill);
  if (c) { ((or_state*)c)->relaxed = h->relaxed; ((or_state*)c)->uni = h->uni; }
  return c;
}
