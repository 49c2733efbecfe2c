/*
 * picasso_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of one Picasso round and of
 * the whole iterative algorithm (Ferdous et al., "Picasso: Memory-Efficient
 * Graph Coloring Using Palettes With Applications in Quantum Computing",
 * arXiv 2401.06713).  Only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark may load this library.  The product (the CUDA
 * library) never links, calls or reads anything here, and nothing here is
 * shared with it: the Pauli predicate uses the paper's 3-bit code instead of
 * the product's symplectic words, and Philox / Floyd are written out again.
 *
 * Every function follows a passage of the paper (section / algorithm /
 * equation given beside it) or a published definition it relies on.  There
 * is no blocking, fusion or reordering beyond what those definitions state;
 * threads are used only over independent rows of the conflict graph.
 *
 * Readings where the paper is silent (they bind product and oracle alike):
 *   - the colored graph is the complement G' of the anticommutation graph:
 *     u != v are adjacent iff they commute (Sec. II, Def. 1 and the complement
 *     construction; Sec. III-A "in our case, a non-edge");
 *   - P_l = max(1, ceil(n_l * num / den)), L_l = min(P_l, max(1,
 *     ceil(alpha * ln n_l))) (Table I: P a fraction of |V|, L = alpha log|V|);
 *   - palette of round l is [base_l, base_l + P_l), base_l = sum of earlier
 *     P (Alg. 1 text: colors of a round are never reused later);
 *   - a list is L distinct colors drawn uniformly (Floyd's sampling), sorted;
 *   - conflict coloring is the static Random order of Sec. III-B with
 *     first-fit: vertices in ascending (priority, global id) order take the
 *     smallest list color not used by an already-colored conflict neighbour;
 *     unconflicted vertices therefore get their smallest list color;
 *   - conflict rows are stored "color-major": row u lists, for each color c
 *     of u's list in ascending order, the neighbours v that also hold c, in
 *     ascending v; an edge whose lists share m colors appears in m runs of
 *     each of its two rows (the coloring step tests color c against exactly
 *     the run of c).
 *
 * Parity pins (what fixes this file against something other than itself) are
 * in the test-suite: Philox known-answer vectors, the 16-entry Pauli truth
 * table, the complete-4^q degree invariant, brute force over character
 * strings, exact Floyd distributions and the closed-form conflict count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_LIST 1u
#define ORC_TAG_PRIO 2u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel Random   */
/* Numbers: As Easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 bit      */
/* multiplies; the key is bumped by the Weyl constants between rounds.       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* The i-th 32-bit draw of stream (seed, round, gid, tag): counter word 0/1 =
 * gid, word 2 = round, word 3 = tag << 24 | block, block = i / 4.           */
static uint32_t orc_draw(uint64_t seed, int32_t round, int64_t gid,
                         uint32_t tag, uint32_t i) {
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = (uint32_t)((uint64_t)gid & 0xffffffffu);
  ctr[1] = (uint32_t)((uint64_t)gid >> 32);
  ctr[2] = (uint32_t)round;
  ctr[3] = (tag << 24) | (i / 4u);
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, out);
  return out[i % 4u];
}

uint32_t orc_draw_u32(uint64_t seed, int32_t round, int64_t gid, uint32_t tag,
                      uint32_t i) {
  return orc_draw(seed, round, gid, tag, i);
}

/* Priority of a vertex in round l: first draw of its PRIO stream.  The
 * coloring order is ascending (priority, gid).                             */
uint32_t orc_priority(uint64_t seed, int32_t round, int64_t gid) {
  return orc_draw(seed, round, gid, ORC_TAG_PRIO, 0u);
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Alg. 1 assign_rand_list_colors for one vertex: L distinct colors drawn
 * uniformly from the round palette.  Floyd's sampling (J. Bentley, R. Floyd,
 * "A sample of brilliance", CACM 1987): for j = P-L .. P-1 draw t uniform in
 * [0, j]; keep t unless already kept, in which case keep j.  A draw x maps to
 * [0, j] as floor(x * (j+1) / 2^32).  The list is returned sorted and
 * shifted by base.                                                          */
void orc_draw_list(uint64_t seed, int32_t round, int64_t gid, int64_t P,
                   int32_t L, int64_t base, int64_t* out) {
  int32_t m = 0;
  for (int64_t j = P - L; j < P; ++j) {
    uint32_t x = orc_draw(seed, round, gid, ORC_TAG_LIST, (uint32_t)m);
    int64_t t = (int64_t)(((uint64_t)x * (uint64_t)(j + 1)) >> 32);
    int seen = 0;
    for (int32_t a = 0; a < m; ++a)
      if (out[a] == t) seen = 1;
    out[m++] = seen ? j : t;
  }
  qsort(out, (size_t)L, sizeof(int64_t), cmp_i64);
  for (int32_t a = 0; a < L; ++a) out[a] += base;
}

/* orc_draw_list for many vertices: out[m][L].                               */
void orc_draw_lists_many(uint64_t seed, int32_t round, const int64_t* gids,
                         int64_t m, int64_t P, int32_t L, int64_t base,
                         int64_t* out) {
  for (int64_t i = 0; i < m; ++i)
    orc_draw_list(seed, round, gids[i], P, L, base, out + i * L);
}

void orc_priorities_many(uint64_t seed, int32_t round, const int64_t* gids,
                         int64_t m, uint32_t* out) {
  for (int64_t i = 0; i < m; ++i) out[i] = orc_priority(seed, round, gids[i]);
}

/* ------------------------------------------------------------------------ */
/* Pauli predicate (Sec. III-A).  Characters are codes 0=I 1=X 2=Y 3=Z.      */
/* ------------------------------------------------------------------------ */

/* Direct statement: two strings anticommute iff an odd number of positions
 * hold two different non-identity Paulis.  Returns 1 if they commute.      */
int orc_commute_chars(const uint8_t* a, const uint8_t* b, int32_t q) {
  int count = 0;
  for (int32_t i = 0; i < q; ++i)
    if (a[i] != 0 && b[i] != 0 && a[i] != b[i]) ++count;
  return (count % 2) == 0;
}

/* The paper's "inverse one-hot" code: X=110, Y=101, Z=011, I=000, ten
 * characters per 32-bit word (character i of a word in bits 3i..3i+2).    */
static uint32_t orc_code3(uint8_t ch) {
  switch (ch) {
    case 1: return 6u; /* X = 110 */
    case 2: return 5u; /* Y = 101 */
    case 3: return 3u; /* Z = 011 */
    default: return 0u; /* I = 000 */
  }
}

int32_t orc_words3(int32_t q) { return (q + 9) / 10; }

void orc_encode3(const uint8_t* chars, int64_t n, int32_t q, uint32_t* enc) {
  int32_t w3 = orc_words3(q);
  for (int64_t v = 0; v < n; ++v) {
    for (int32_t w = 0; w < w3; ++w) enc[v * w3 + w] = 0u;
    for (int32_t i = 0; i < q; ++i)
      enc[v * w3 + i / 10] |= orc_code3(chars[v * (int64_t)q + i]) << (3 * (i % 10));
  }
}

/* Number of one bits of x (the compiler's population count builtin). */
static int orc_popcount32(uint32_t x) { return __builtin_popcount(x); }

/* AND the codes and count ones: the count's parity is the parity of the
 * number of mismatching non-identity positions.  Returns 1 if they commute. */
int orc_commute3(const uint32_t* a, const uint32_t* b, int32_t w3) {
  int ones = 0;
  for (int32_t w = 0; w < w3; ++w) ones += orc_popcount32(a[w] & b[w]);
  return (ones % 2) == 0;
}

/* Index in a of the smallest color in both sorted lists, or -1 if they are
 * disjoint (Sec. III-A: with sorted lists the test takes O(L)).             */
static int32_t orc_min_shared_index(const int64_t* a, const int64_t* b, int32_t L) {
  int32_t i = 0, j = 0;
  while (i < L && j < L) {
    if (a[i] == b[j]) return i;
    if (a[i] < b[j])
      ++i;
    else
      ++j;
  }
  return -1;
}

int64_t orc_min_shared(const int64_t* a, const int64_t* b, int32_t L) {
  int32_t i = orc_min_shared_index(a, b, L);
  return i < 0 ? -1 : a[i];
}

/* ------------------------------------------------------------------------ */
/* Conflict graph (Alg. 1 construct_conflict_graph; Sec. III-A).            */
/* ------------------------------------------------------------------------ */

/* One row in color-major order.  enc: [n][w3] codes of the round's vertices
 * (round-local ids), lists: [n][L] sorted colors, all in [cmin, cmin +
 * ncol).  Row u lists, for each color c_k of u's list (ascending k), every
 * other vertex v that commutes with u and also holds c_k, ascending in v; a
 * neighbour sharing m colors with u therefore appears in m of u's runs.
 * Writes the row into out (may be NULL to count) and returns its length.
 * Scratch (per calling thread): idx [ncol] all zero on entry and on return
 * (idx[c - cmin] = k + 1 while c is u's k-th color); cnt [L + 1]; hit_k /
 * hit_v a growable list of the row's (k, v) hits in the order found
 * (ascending v), which a counting sort by k turns into the runs.           */
typedef struct {
  int32_t* idx;
  int64_t cmin, ncol;
  int64_t* cnt;
  int32_t* hit_k;
  int32_t* hit_v;
  int64_t cap;
} orc_row_scratch;

static void orc_hit(orc_row_scratch* sc, int64_t len, int32_t k, int64_t v) {
  if (len == sc->cap) {
    sc->cap = sc->cap ? 2 * sc->cap : 1024;
    sc->hit_k = (int32_t*)realloc(sc->hit_k, sizeof(int32_t) * (size_t)sc->cap);
    sc->hit_v = (int32_t*)realloc(sc->hit_v, sizeof(int32_t) * (size_t)sc->cap);
  }
  sc->hit_k[len] = k;
  sc->hit_v[len] = (int32_t)v;
}

/* The row's (k, v) hits into the scratch list, in ascending v; sc->cnt[k+1]
 * counts the hits of u's k-th color.  Returns the count.                   */
static int64_t orc_conflict_hits(int64_t u, int64_t n, const uint32_t* enc, int32_t w3,
                                 const int64_t* lists, int32_t L, orc_row_scratch* sc) {
  const int64_t* a = lists + u * L;
  for (int32_t k = 0; k < L; ++k) sc->idx[a[k] - sc->cmin] = k + 1;
  for (int32_t k = 0; k <= L; ++k) sc->cnt[k] = 0;
  int64_t len = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (v == u) continue;
    if (!orc_commute3(enc + u * w3, enc + v * w3, w3)) continue;
    const int64_t* b = lists + v * L;
    for (int32_t j = 0; j < L; ++j) {
      int32_t k1 = sc->idx[b[j] - sc->cmin]; /* b[j] is u's color k1 - 1 */
      if (k1 == 0) continue;
      sc->cnt[k1]++;
      orc_hit(sc, len++, k1 - 1, v);
    }
  }
  for (int32_t k = 0; k < L; ++k) sc->idx[a[k] - sc->cmin] = 0;
  return len;
}

/* Lays the hits out as runs in ascending k (a counting sort by k; inside a
 * run the hits keep their ascending v).                                    */
static void orc_conflict_layout(orc_row_scratch* sc, int64_t len, int32_t L, int32_t* out) {
  int64_t run = 0;
  for (int32_t k = 1; k <= L; ++k) {
    int64_t c = sc->cnt[k];
    sc->cnt[k] = run;
    run += c;
  }
  for (int64_t h = 0; h < len; ++h) out[sc->cnt[sc->hit_k[h] + 1]++] = sc->hit_v[h];
}

int64_t orc_conflict_row(int64_t u, int64_t n, const uint32_t* enc, int32_t w3,
                         const int64_t* lists, int32_t L, orc_row_scratch* sc,
                         int32_t* out) {
  int64_t len = orc_conflict_hits(u, n, enc, w3, lists, L, sc);
  if (out) orc_conflict_layout(sc, len, L, out);
  return len;
}

/* The paper's conflict graph G_c with each edge once (Sec. III-A: u and v
 * are adjacent iff they commute and their lists share a color): the
 * partners v > u of u, ascending, into the scratch hit list (hit_v).
 * Returns the count.                                                       */
static int64_t orc_edge_row(int64_t u, int64_t n, const uint32_t* enc, int32_t w3,
                            const int64_t* lists, int32_t L, orc_row_scratch* sc) {
  const int64_t* a = lists + u * L;
  for (int32_t k = 0; k < L; ++k) sc->idx[a[k] - sc->cmin] = k + 1;
  int64_t len = 0;
  for (int64_t v = u + 1; v < n; ++v) {
    if (!orc_commute3(enc + u * w3, enc + v * w3, w3)) continue;
    const int64_t* b = lists + v * L;
    int meet = 0;
    for (int32_t j = 0; j < L; ++j)
      if (sc->idx[b[j] - sc->cmin]) meet = 1;
    if (meet) orc_hit(sc, len++, 0, v);
  }
  for (int32_t k = 0; k < L; ++k) sc->idx[a[k] - sc->cmin] = 0;
  return len;
}

typedef struct {
  int64_t n, r0, r1, stride;
  const uint32_t* enc;
  int32_t w3;
  const int64_t* lists;
  int32_t L;
  const int64_t* rows; /* NULL: rows 0..count-1 themselves */
  int64_t cmin, ncol;  /* every list color lies in [cmin, cmin + ncol) */
  int64_t* lens;
  const int64_t* off;
  int32_t* col;
  int32_t** rowbuf; /* non-NULL: each row into its own malloc'd buffer */
  int32_t edges;    /* 1: the deduplicated edge rows of orc_edge_row instead */
} orc_rows_job;

static void* orc_rows_worker(void* arg) {
  orc_rows_job* j = (orc_rows_job*)arg;
  orc_row_scratch sc;
  memset(&sc, 0, sizeof(sc));
  sc.cmin = j->cmin;
  sc.ncol = j->ncol;
  sc.idx = (int32_t*)calloc((size_t)(j->ncol > 0 ? j->ncol : 1), sizeof(int32_t));
  sc.cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(j->L + 2));
  for (int64_t i = j->r0; i < j->r1; i += j->stride) {
    int64_t u = j->rows ? j->rows[i] : i;
    if (j->rowbuf) {
      /* the row goes to the scratch hit list first, then to a buffer of its own */
      int64_t len = j->edges ? orc_edge_row(u, j->n, j->enc, j->w3, j->lists, j->L, &sc)
                             : orc_conflict_hits(u, j->n, j->enc, j->w3, j->lists, j->L, &sc);
      int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
      if (j->edges)
        memcpy(tmp, sc.hit_v, sizeof(int32_t) * (size_t)len);
      else
        orc_conflict_layout(&sc, len, j->L, tmp);
      j->rowbuf[i] = tmp;
      j->lens[i] = len;
      continue;
    }
    int32_t* dst = j->col ? j->col + j->off[i] : NULL;
    int64_t len = orc_conflict_row(u, j->n, j->enc, j->w3, j->lists, j->L, &sc, dst);
    if (j->lens) j->lens[i] = len;
  }
  free(sc.idx);
  free(sc.cnt);
  free(sc.hit_k);
  free(sc.hit_v);
  return NULL;
}

static void orc_run_rows(orc_rows_job proto, int64_t count, int32_t threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  const int64_t E = proto.n * proto.L;
  int64_t lo = E > 0 ? proto.lists[0] : 0, hi = E > 0 ? proto.lists[0] : -1;
  for (int64_t e = 1; e < E; ++e) {
    if (proto.lists[e] < lo) lo = proto.lists[e];
    if (proto.lists[e] > hi) hi = proto.lists[e];
  }
  proto.cmin = lo;
  proto.ncol = hi - lo + 1;
  pthread_t tid[256];
  orc_rows_job jobs[256];
  for (int32_t t = 0; t < threads; ++t) {
    jobs[t] = proto;
    jobs[t].r0 = t;
    jobs[t].r1 = count;
    jobs[t].stride = threads;
    pthread_create(&tid[t], NULL, orc_rows_worker, &jobs[t]);
  }
  for (int32_t t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
}

/* Selected rows (round-local ids rows[0..m)) of the conflict graph.  With
 * col == NULL only lens is filled; otherwise off[m] gives where each row
 * goes.                                                                    */
void orc_conflict_rows(int64_t n, const uint32_t* enc, int32_t w3,
                       const int64_t* lists, int32_t L, const int64_t* rows,
                       int64_t m, int64_t* lens, const int64_t* off,
                       int32_t* col, int32_t threads) {
  orc_rows_job p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.enc = enc;
  p.w3 = w3;
  p.lists = lists;
  p.L = L;
  p.rows = rows;
  p.lens = lens;
  p.off = off;
  p.col = col;
  orc_run_rows(p, m, threads);
}

/* Whole CSR: row lengths, then off[n+1] (int64) and col.                   */
int64_t orc_conflict_nnz(int64_t n, const uint32_t* enc, int32_t w3,
                         const int64_t* lists, int32_t L, int64_t* lens,
                         int32_t threads) {
  orc_conflict_rows(n, enc, w3, lists, L, NULL, n, lens, NULL, NULL, threads);
  int64_t s = 0;
  for (int64_t u = 0; u < n; ++u) s += lens[u];
  return s;
}

void orc_conflict_fill(int64_t n, const uint32_t* enc, int32_t w3,
                       const int64_t* lists, int32_t L, const int64_t* lens,
                       int64_t* off, int32_t* col, int32_t threads) {
  off[0] = 0;
  for (int64_t u = 0; u < n; ++u) off[u + 1] = off[u] + lens[u];
  orc_conflict_rows(n, enc, w3, lists, L, NULL, n, NULL, off, col, threads);
}

/* Rows rows[0..m) (NULL: all n rows) in one pass: off[m+1] receives the
 * offsets and *col a malloc'd array of the concatenated rows (release it
 * with orc_free).  edges = 0: the color-major rows of orc_conflict_row;
 * edges = 1: the deduplicated rows of orc_edge_row (partners v > u).
 * Returns the total length.                                               */
int64_t orc_conflict_collect(int64_t n, const uint32_t* enc, int32_t w3, const int64_t* lists, int32_t L,
                             const int64_t* rows, int64_t m, int32_t edges, int32_t threads, int64_t* off,
                             int32_t** col) {
  int32_t** rowbuf = (int32_t**)malloc(sizeof(int32_t*) * (size_t)(m > 0 ? m : 1));
  int64_t* lens = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  orc_rows_job p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.enc = enc;
  p.w3 = w3;
  p.lists = lists;
  p.L = L;
  p.rows = rows;
  p.lens = lens;
  p.rowbuf = rowbuf;
  p.edges = edges;
  orc_run_rows(p, m, threads);
  off[0] = 0;
  for (int64_t i = 0; i < m; ++i) off[i + 1] = off[i] + lens[i];
  int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[m] > 0 ? off[m] : 1));
  for (int64_t i = 0; i < m; ++i) {
    memcpy(out + off[i], rowbuf[i], sizeof(int32_t) * (size_t)lens[i]);
    free(rowbuf[i]);
  }
  free(rowbuf);
  free(lens);
  *col = out;
  return off[m];
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Coloring of the conflict graph: static Random order, first fit (Sec.      */
/* III-B "static order schemes"; Alg. 1 color_unconflicted_vertices and      */
/* color_conflict_graph).                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t key;
  int64_t v;
} orc_key;

static int cmp_key(const void* a, const void* b) {
  uint64_t x = ((const orc_key*)a)->key, y = ((const orc_key*)b)->key;
  return (x > y) - (x < y);
}

/* gids[n]: global ids of the round's vertices (round-local id = index).
 * color_local[n] receives the global color or -1.  Returns colored count.  */
int64_t orc_color_greedy(uint64_t seed, int32_t round, int64_t n,
                         const int64_t* gids, const int64_t* lists, int32_t L,
                         const int64_t* off, const int32_t* col, int64_t P,
                         int64_t base, int64_t* color_local) {
  orc_key* order = (orc_key*)malloc(sizeof(orc_key) * (size_t)(n > 0 ? n : 1));
  int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
  for (int64_t c = 0; c < P; ++c) stamp[c] = -1;
  for (int64_t v = 0; v < n; ++v) {
    uint64_t pr = orc_priority(seed, round, gids[v]);
    order[v].key = (pr << 32) | (uint64_t)(uint32_t)gids[v];
    order[v].v = v;
    color_local[v] = -1;
  }
  qsort(order, (size_t)n, sizeof(orc_key), cmp_key);
  int64_t colored = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = order[i].v;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      int64_t cu = color_local[col[e]];
      if (cu >= 0) stamp[cu - base] = v;
    }
    for (int32_t k = 0; k < L; ++k) {
      int64_t c = lists[v * L + k];
      if (stamp[c - base] != v) {
        color_local[v] = c;
        ++colored;
        break;
      }
    }
  }
  free(order);
  free(stamp);
  return colored;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: dynamic greedy list coloring of G_c (Sec. III-B "dynamic vertex   */
/* order scheme").  Vertices sit in buckets by the size of their remaining   */
/* list; the lowest bucket is served first; the chosen vertex takes a color  */
/* drawn uniformly from its remaining list, and that color leaves the lists  */
/* of its uncolored neighbours (a list that becomes empty leaves the vertex  */
/* uncolored).  Readings: "a vertex chosen uniformly at random from the      */
/* lowest bucket" is the bucket's vertex of smallest (priority, gid), the    */
/* priority being the round's Philox priority (for iid priorities, a uniform */
/* pick); "a color chosen uniformly at random" is the remaining list's entry */
/* at floor(x * size / 2^32), x = word 0 of the Philox stream (seed, round,  */
/* gid, tag 4), one draw per vertex.                                         */
/* ------------------------------------------------------------------------ */
static int64_t orc_dyn_pick(uint64_t seed, int32_t round, int64_t gid, const int64_t* rem, int32_t L,
                            const int8_t* alive) {
  int32_t size = 0;
  for (int32_t k = 0; k < L; ++k) size += alive[k];
  uint32_t x = orc_draw_u32(seed, round, gid, 4u, 0u);
  int32_t idx = (int32_t)(((uint64_t)x * (uint64_t)size) >> 32);
  for (int32_t k = 0; k < L; ++k) {
    if (!alive[k]) continue;
    if (idx == 0) return rem[k];
    --idx;
  }
  return -1;
}

/* remove color c from u's remaining list; returns 1 if it was there */
static int orc_dyn_remove(const int64_t* list_u, int8_t* alive_u, int32_t L, int64_t c) {
  for (int32_t k = 0; k < L; ++k)
    if (alive_u[k] && list_u[k] == c) {
      alive_u[k] = 0;
      return 1;
    }
  return 0;
}

typedef struct {
  int32_t size;
  uint64_t key; /* priority << 32 | gid */
  int64_t v;
} orc_dyn_entry;

static int orc_dyn_less(const orc_dyn_entry* a, const orc_dyn_entry* b) {
  if (a->size != b->size) return a->size < b->size;
  return a->key < b->key;
}

/* Sequential Alg. 2.  off/col: the two-sided per-color rows of G_c (any
 * neighbour order; repeats harmless).  color_local[n]: color or -1.
 * Returns the colored count.  The "lowest bucket, then smallest key" choice
 * is served by a binary heap of (size, key) entries; an entry whose size is
 * stale or whose vertex is done is skipped when popped.                    */
int64_t orc_color_dynamic(uint64_t seed, int32_t round, int64_t n, const int64_t* gids, const int64_t* lists,
                          int32_t L, const int64_t* off, const int32_t* col, int64_t* color_local) {
  int8_t* alive = (int8_t*)malloc((size_t)(n * L + 1));
  int32_t* size = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int8_t* done = (int8_t*)malloc((size_t)(n + 1));
  int64_t cap = n + 1 + 64;
  orc_dyn_entry* heap = (orc_dyn_entry*)malloc(sizeof(orc_dyn_entry) * (size_t)cap);
  int64_t hn = 0;
#define ORC_PUSH(E)                                                                            \
  do {                                                                                         \
    if (hn == cap) {                                                                           \
      cap *= 2;                                                                                \
      heap = (orc_dyn_entry*)realloc(heap, sizeof(orc_dyn_entry) * (size_t)cap);               \
    }                                                                                          \
    int64_t i_ = hn++;                                                                         \
    heap[i_] = (E);                                                                            \
    while (i_ > 0 && orc_dyn_less(&heap[i_], &heap[(i_ - 1) / 2])) {                           \
      orc_dyn_entry t_ = heap[i_];                                                             \
      heap[i_] = heap[(i_ - 1) / 2];                                                           \
      heap[(i_ - 1) / 2] = t_;                                                                 \
      i_ = (i_ - 1) / 2;                                                                       \
    }                                                                                          \
  } while (0)
  for (int64_t v = 0; v < n; ++v) {
    for (int32_t k = 0; k < L; ++k) alive[v * L + k] = 1;
    size[v] = L;
    done[v] = 0;
    color_local[v] = -1;
    orc_dyn_entry e = {L, ((uint64_t)orc_priority(seed, round, gids[v]) << 32) | (uint32_t)gids[v], v};
    ORC_PUSH(e);
  }
  int64_t colored = 0;
  while (hn > 0) {
    orc_dyn_entry top = heap[0];
    heap[0] = heap[--hn];
    for (int64_t i = 0;;) {
      int64_t l = 2 * i + 1, r = l + 1, m = i;
      if (l < hn && orc_dyn_less(&heap[l], &heap[m])) m = l;
      if (r < hn && orc_dyn_less(&heap[r], &heap[m])) m = r;
      if (m == i) break;
      orc_dyn_entry t = heap[i];
      heap[i] = heap[m];
      heap[m] = t;
      i = m;
    }
    const int64_t v = top.v;
    if (done[v] || top.size != size[v]) continue;
    done[v] = 1;
    const int64_t c = orc_dyn_pick(seed, round, gids[v], lists + v * L, L, alive + v * L);
    color_local[v] = c;
    ++colored;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      const int64_t u = col[e];
      if (done[u]) continue;
      if (!orc_dyn_remove(lists + u * L, alive + u * L, L, c)) continue;
      if (--size[u] == 0) {
        done[u] = 1; /* no color left: stays uncolored */
        continue;
      }
      orc_dyn_entry eu = {size[u], ((uint64_t)orc_priority(seed, round, gids[u]) << 32) | (uint32_t)gids[u], u};
      ORC_PUSH(eu);
    }
  }
#undef ORC_PUSH
  free(alive);
  free(size);
  free(done);
  free(heap);
  return colored;
}

/* The parallel form of Alg. 2's rule (what the GPU computes): in each step
 * every uncolored vertex with a nonempty list whose (size, priority, gid) is
 * smaller than that of each such neighbour takes its color (the same draw as
 * above), then all those colors leave the neighbours' lists; a vertex whose
 * list empties is left uncolored at the start of the next step.  Returns the
 * colored count; *steps gets the number of steps.                          */
int64_t orc_color_dynamic_par(uint64_t seed, int32_t round, int64_t n, const int64_t* gids, const int64_t* lists,
                              int32_t L, const int64_t* off, const int32_t* col, int64_t* color_local,
                              int64_t* steps) {
  int8_t* alive = (int8_t*)malloc((size_t)(n * L + 1));
  int32_t* size = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int8_t* state = (int8_t*)malloc((size_t)(n + 1)); /* 0 active, 1 colored, 2 left uncolored */
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
  int8_t* pick = (int8_t*)malloc((size_t)(n + 1));
  for (int64_t v = 0; v < n; ++v) {
    for (int32_t k = 0; k < L; ++k) alive[v * L + k] = 1;
    size[v] = L;
    state[v] = 0;
    color_local[v] = -1;
    key[v] = ((uint64_t)orc_priority(seed, round, gids[v]) << 32) | (uint32_t)gids[v];
  }
  int64_t colored = 0, t = 0, active = n;
  while (active > 0) {
    ++t;
    for (int64_t v = 0; v < n; ++v)
      if (state[v] == 0 && size[v] == 0) state[v] = 2;
    for (int64_t v = 0; v < n; ++v) {
      pick[v] = 0;
      if (state[v] != 0) continue;
      int ok = 1;
      for (int64_t e = off[v]; e < off[v + 1] && ok; ++e) {
        const int64_t u = col[e];
        if (state[u] != 0) continue;
        if (size[u] < size[v] || (size[u] == size[v] && key[u] < key[v])) ok = 0;
      }
      pick[v] = (int8_t)ok;
    }
    for (int64_t v = 0; v < n; ++v) {
      if (!pick[v]) continue;
      color_local[v] = orc_dyn_pick(seed, round, gids[v], lists + v * L, L, alive + v * L);
      state[v] = 1;
      ++colored;
    }
    for (int64_t v = 0; v < n; ++v) {
      if (!pick[v]) continue;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        const int64_t u = col[e];
        if (state[u] == 0 && orc_dyn_remove(lists + u * L, alive + u * L, L, color_local[v])) --size[u];
      }
    }
    active = 0;
    for (int64_t v = 0; v < n; ++v) active += state[v] == 0;
  }
  if (steps) *steps = t;
  free(alive);
  free(size);
  free(state);
  free(key);
  free(pick);
  return colored;
}

/* Round parameters (Table I; Sec. VI "P a percentage of |V|, L = alpha
 * log|V|, the same percentage and alpha in every iteration").              */
void orc_round_params(int64_t n, int64_t num, int64_t den, double alpha,
                      int64_t* P, int32_t* L) {
  int64_t p = (n * num + den - 1) / den;
  if (p < 1) p = 1;
  double l = ceil(alpha * log((double)n));
  int64_t li = (int64_t)l;
  if (li < 1) li = 1;
  if (li > p) li = p;
  *P = p;
  *L = (int32_t)li;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: the whole iterative algorithm.                                    */
/* chars [N][q]; color[N] receives global colors.  Per-round statistics      */
/* (n, P, L, base, nnz, colored) go to stats[6 * r] for r < max_rounds.      */
/* Returns the number of rounds run, or -1 if max_rounds was hit first.      */
/* ------------------------------------------------------------------------ */
int32_t orc_run_colorer(const uint8_t* chars, int64_t N, int32_t q, uint64_t seed, int64_t num, int64_t den,
                        double alpha, int32_t max_rounds, int32_t threads, int32_t colorer, int64_t* color,
                        int64_t* stats);

int32_t orc_run(const uint8_t* chars, int64_t N, int32_t q, uint64_t seed,
                int64_t num, int64_t den, double alpha, int32_t max_rounds,
                int32_t threads, int64_t* color, int64_t* stats) {
  return orc_run_colorer(chars, N, q, seed, num, den, alpha, max_rounds, threads, 0, color, stats);
}

/* colorer: 0 static Random order with first fit (the default), 1 Alg. 2
 * sequential, 2 Alg. 2's parallel rule.                                    */
int32_t orc_run_colorer(const uint8_t* chars, int64_t N, int32_t q, uint64_t seed, int64_t num, int64_t den,
                        double alpha, int32_t max_rounds, int32_t threads, int32_t colorer, int64_t* color,
                        int64_t* stats) {
  int32_t w3 = orc_words3(q);
  uint32_t* enc_all = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N * w3 + 1));
  orc_encode3(chars, N, q, enc_all);
  for (int64_t v = 0; v < N; ++v) color[v] = -1;
  int64_t* gids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
  int64_t n = N;
  for (int64_t v = 0; v < N; ++v) gids[v] = v;
  int64_t base = 0;
  int32_t round = 1;
  while (n > 0) {
    if (round > max_rounds) {
      free(enc_all);
      free(gids);
      return -1;
    }
    int64_t P;
    int32_t L;
    orc_round_params(n, num, den, alpha, &P, &L);
    uint32_t* enc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n * w3 + 1));
    int64_t* lists = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * L + 1));
    for (int64_t v = 0; v < n; ++v) {
      memcpy(enc + v * w3, enc_all + gids[v] * w3, sizeof(uint32_t) * (size_t)w3);
      orc_draw_list(seed, round, gids[v], P, L, base, lists + v * L);
    }
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* col = NULL;
    int64_t nnz = orc_conflict_collect(n, enc, w3, lists, L, NULL, n, 0, threads, off, &col);
    int64_t* cl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t colored =
        colorer == 1   ? orc_color_dynamic(seed, round, n, gids, lists, L, off, col, cl)
        : colorer == 2 ? orc_color_dynamic_par(seed, round, n, gids, lists, L, off, col, cl, NULL)
                       : orc_color_greedy(seed, round, n, gids, lists, L, off, col, P, base, cl);
    if (stats) {
      int64_t* s = stats + 6 * (round - 1);
      s[0] = n;
      s[1] = P;
      s[2] = L;
      s[3] = base;
      s[4] = nnz;
      s[5] = colored;
    }
    /* Alg. 1, end of an iteration: carry the uncolored vertices (ascending gid). */
    int64_t m = 0;
    for (int64_t v = 0; v < n; ++v) {
      if (cl[v] >= 0)
        color[gids[v]] = cl[v];
      else
        gids[m++] = gids[v];
    }
    n = m;
    base += P;
    ++round;
    free(enc);
    free(lists);
    free(off);
    free(col);
    free(cl);
  }
  free(enc_all);
  free(gids);
  return round - 1;
}

/* ------------------------------------------------------------------------ */
/* Instance features for the parameter regressor of Sec. V.  The paper feeds */
/* its regressor (beta, |V|, |E|); here the inputs are the size, the qubit   */
/* count, the mean Pauli weight, a sampled commuting fraction (the edge      */
/* density of G') and the memory budget.  This part counts:                  */
/*   out[0] = non-identity characters over all n strings                     */
/*   out[1] = commuting pairs among `samples` pairs of distinct strings; pair */
/*            p takes draws 0 and 1 of stream (seed, round 0, gid p, tag 3): */
/*            first string floor(d0 n / 2^32), second floor(d1 (n-1) / 2^32), */
/*            plus one when not below the first.                              */
/* ------------------------------------------------------------------------ */
void orc_feature_counts(const uint8_t* chars, int64_t n, int32_t q, uint64_t seed,
                        int64_t samples, int64_t out[2]) {
  int64_t weight = 0, commuting = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int32_t i = 0; i < q; ++i) weight += chars[v * (int64_t)q + i] != 0;
  if (n < 2) samples = 0;
  for (int64_t p = 0; p < samples; ++p) {
    uint32_t d0 = orc_draw(seed, 0, p, 3u, 0u), d1 = orc_draw(seed, 0, p, 3u, 1u);
    int64_t a = (int64_t)(((uint64_t)d0 * (uint64_t)n) >> 32);
    int64_t b = (int64_t)(((uint64_t)d1 * (uint64_t)(n - 1)) >> 32);
    if (b >= a) ++b;
    commuting += orc_commute_chars(chars + a * (int64_t)q, chars + b * (int64_t)q, q);
  }
  out[0] = weight;
  out[1] = commuting;
}
