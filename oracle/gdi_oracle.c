/*
 * gdi_oracle.c -- plain, slow, sequential CPU oracle for the Globally Decoupled Ising (GDI)
 * balanced min-cut annealer (Cook, Jin, Tan, arXiv:1908.00210).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it. It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (each function names the passage it follows):
 *   - the min-cut Ising energy  H = H_A + H_B,  H_A = A (sum_i s_i)^2,
 *     H_B = B * sum_<ij> w_ij (1 - s_i s_j)/2                     (Eq. 4, 5, 6)
 *   - the energy change of one spin flip given the exact magnetisation G = sum s
 *       dE_i = B s_i h_i + 4A (1 - s_i G),  h_i = sum_j w_ij s_j     (Eq. 4-6; Alg. 3 argmin term,
 *                                                                    read with G counting the
 *                                                                    other spins, see below)
 *   - Algorithm 3 (GDI): G is computed once before the first sweep and then updated by the
 *     change of each flipped spin; every spin decides from G and its neighbours only.
 *   - the noise: a per-temperature integer acceptance threshold table (Metropolis form, or the
 *     paper's argmin-then-random-flip-with-P_f form, Section 5.2 and Alg. 2/3), drawn with the
 *     counter-based Philox4x32-10 generator (Salmon et al., SC'11) in place of cuRAND.
 *
 * Readings of the paper taken here (the paper leaves these open or garbles them):
 *   R1  Alg. 3's "argmin(H_B + A(G + s_i)^2)" is read with G = sum over the OTHER spins, which
 *       gives the exact flip cost 4A(1 - s_i G) for the balance term; "atomicAdd(G + s_i)" is read
 *       as adding the change of s_i (+-2 or 0), so G stays exact after every update.
 *   R2  Determinism in place of the GPU race: vertices are updated colour class by colour class
 *       (a class has no internal edges, so every h_i inside a class is fixed while the class is
 *       updated); inside a class the rank order is that of splitmix64(vertex id), a fixed
 *       pseudo-random order.  A class is cut into windows of W consecutive ranks (W = 0: the whole
 *       class).
 *       Inside a window every spin sees the exact running G, in a canonical order: first the
 *       spins that were +1 at window start, sorted by their flip threshold gamma ascending (rank
 *       ascending on ties), then the spins that were -1, sorted by gamma' descending (rank
 *       ascending); on odd sweeps the -1 group goes first.  gamma is the smallest G at which the
 *       spin's draw accepts the flip, so the spins that most want to flip get to the running G
 *       first, the way the earliest atomics would.  gamma only fixes that order: each flip is
 *       decided from its definition, the draw against the table entry of the energy change at
 *       the running G, and the run counts any flip where "G >= gamma" would have said otherwise
 *       (there must be none).
 *   R3  One draw per spin per sweep merges "argmin" and "flip with probability P_f" into a single
 *       Bernoulli decision with the same probabilities (flip w.p. 1-P_f if dE<0, 1/2 if dE=0, P_f
 *       if dE>0); "flip iff u <= P_f" (Section 5.2) becomes u32 < floor(P_f 2^32) + 1.
 *   R4  Balanced random initial spins: ranks are paired (2p, 2p+1) and a Philox coin gives the
 *       pair (+1,-1) or (-1,+1); an odd last rank starts at -1.
 *   R5  After the last sweep an exact-balance repair flips the k = (|G| - (n mod 2))/2 majority
 *       spins with the smallest (s_i h_i, rank) keys.
 *   Stale option (the racy variant's reference): every spin of a window decides on the G of the
 *       window start, as parallel threads that all read G before any flip of the window lands
 *       (Section 5.3's outdated G); the flips still update G exactly afterwards.
 *
 * Everything is integer except the threshold table, which is built in double precision with
 * exp() and pow() from libm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_COLOR -2
#define ORC_ERR_OOM -3
#define ORC_ERR_RANGE -4

#define ORC_METROPOLIS 0
#define ORC_PAPER_PF 1

#define INF64 ((int64_t)1 << 62)

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10, written from the published description (Salmon, Moraes, Dror, Shaw, SC'11):
 * ten rounds of two 32x32->64 multiplies with fixed multipliers, a Feistel-like word exchange
 * and a Weyl-sequence key schedule.                                                          */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

/* Philox4x32-10 of n counters under one key (out[4 i .. 4 i + 3] for ctr[4 i .. 4 i + 3]). */
void oracle_philox4x32_10_many(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* One 32-bit draw: counter (c0, c1, c2, c3), key = (seed low word, seed high word), word w. */
static uint32_t draw_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int w)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[w];
}

/* ------------------------------------------------------------------------------------------ */
/* splitmix64 finaliser (Steele, Lea, Flood, OOPSLA'14), used only for the per-sweep digest.  */
static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t digest_term(int64_t rank, int64_t sweep, int64_t replica)
{
    const uint64_t key = ((uint64_t)rank & 0xFFFFFFFFull) | (((uint64_t)sweep & 0xFFFFull) << 32)
                       | (((uint64_t)replica & 0xFFFFull) << 48);
    return mix64(key);
}

/* ------------------------------------------------------------------------------------------ */
/* Threshold table (replaces "reduce P_f", Alg. 2/3).  Row s covers dE = -Ecap .. Ecap; entry
 * thr[s][dE+Ecap] is a uint64 in [0, 2^32]; a draw u32 accepts the flip iff u32 < thr.         */
static double sched_value(double v0, double v1, int s, int M)
{
    if (M <= 1 || v0 == v1) return v0;
    return v0 * pow(v1 / v0, (double)s / (double)(M - 1));
}

static uint64_t metropolis_thr(int64_t dE, double T)
{
    if (dE <= 0) return (uint64_t)1 << 32;
    return (uint64_t)floor(exp(-(double)dE / T) * 4294967296.0);
}

int oracle_table_ecap(int mode, double t0, double t1, double pf0, double pf1, int M)
{
    if (M < 1) return ORC_ERR_ARG;
    if (mode == ORC_PAPER_PF) {
        if (!(pf0 >= 0 && pf0 < 0.5 && pf1 >= 0 && pf1 < 0.5)) return ORC_ERR_ARG;
        if (pf0 != pf1 && (pf0 <= 0 || pf1 <= 0)) return ORC_ERR_ARG;
        return 1;
    }
    if (mode != ORC_METROPOLIS) return ORC_ERR_ARG;
    if (!(t0 > 0 && t1 > 0)) return ORC_ERR_ARG;
    /* smallest E >= 1 whose threshold is 0 at every temperature of the schedule */
    for (int64_t E = 1; E < (1 << 24); ++E) {
        int all_zero = 1;
        for (int s = 0; s < M && all_zero; ++s)
            if (metropolis_thr(E, sched_value(t0, t1, s, M)) != 0) all_zero = 0;
        if (all_zero) return (int)E;
    }
    return ORC_ERR_RANGE;
}

int oracle_build_table(int mode, double t0, double t1, double pf0, double pf1, int M,
                       int ecap, uint64_t *thr)
{
    const int width = 2 * ecap + 1;
    for (int s = 0; s < M; ++s) {
        for (int k = 0; k < width; ++k) {
            const int64_t dE = (int64_t)k - ecap;
            uint64_t t;
            if (mode == ORC_METROPOLIS) {
                t = metropolis_thr(dE, sched_value(t0, t1, s, M));
            } else {
                const double pf = sched_value(pf0, pf1, s, M);
                uint64_t p = (uint64_t)floor(pf * 4294967296.0) + 1;  /* u <= P_f */
                if (p > ((uint64_t)1 << 32)) p = (uint64_t)1 << 32;
                if (dE > 0) t = p;                                     /* random flip only     */
                else if (dE == 0) t = (uint64_t)1 << 31;              /* tie: coin (Eq. 2)    */
                else t = ((uint64_t)1 << 32) - p;                      /* argmin flip, no undo */
            }
            thr[(size_t)s * width + k] = t;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Greedy first-fit colouring in original id order: each vertex takes the smallest colour not
 * used by an already coloured neighbour.  Returns the number of colours.                     */
int oracle_greedy_color(int32_t n, const int64_t *row_ptr, const int32_t *col, int32_t *color)
{
    int32_t ncol = 0;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 2));
    if (!mark) return ORC_ERR_OOM;
    for (int32_t i = 0; i < n + 2; ++i) mark[i] = -1;
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int32_t u = col[e];
            if (u < v) mark[color[u]] = v;
        }
        int32_t c = 0;
        while (mark[c] == v) ++c;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(mark);
    return ncol;
}

/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int32_t v;
} hash_item;

static int cmp_hash(const void *a, const void *b)
{
    const hash_item *x = (const hash_item *)a, *y = (const hash_item *)b;
    return (x->key > y->key) - (x->key < y->key);
}

typedef struct {
    int64_t key;      /* gamma (or -gamma' for the -1 group) */
    int32_t rank;
} sort_item;

static int cmp_item(const void *a, const void *b)
{
    const sort_item *x = (const sort_item *)a, *y = (const sort_item *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->rank > y->rank) - (x->rank < y->rank);
}

static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}
static int64_t ceil_div(int64_t a, int64_t b) /* b > 0 */
{
    return -floor_div(-a, b);
}

/* E*(u): the largest clamped dE that the draw u accepts in table row `row`.
 * Returns -INF64 if none, +INF64 if all (including dE = +Ecap).                              */
static int64_t estar(const uint64_t *row, int ecap, uint32_t u)
{
    int cnt = 0;
    while (cnt < 2 * ecap + 1 && row[cnt] > (uint64_t)u) ++cnt;  /* rows are non-increasing */
    if (cnt == 0) return -INF64;
    if (cnt == 2 * ecap + 1) return INF64;
    return (int64_t)cnt - 1 - ecap;
}

/* Flip threshold of a +1 spin: it flips iff G >= gamma (Eq. 4-6 with R1). */
static int64_t gamma_plus(int64_t h, int64_t Es, int64_t A, int64_t B)
{
    if (Es == -INF64) return INF64;
    if (Es == INF64) return -INF64;
    if (A == 0) return (B * h <= Es) ? -INF64 : INF64;
    return ceil_div(B * h + 4 * A - Es, 4 * A);
}
/* Flip threshold of a -1 spin: it flips iff G <= gamma'. */
static int64_t gamma_minus(int64_t h, int64_t Es, int64_t A, int64_t B)
{
    if (Es == -INF64) return -INF64;
    if (Es == INF64) return INF64;
    if (A == 0) return (-B * h <= Es) ? INF64 : -INF64;
    return floor_div(Es + B * h - 4 * A, 4 * A);
}

typedef struct {
    int32_t n;
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *w;          /* NULL = unit weights */
    const int32_t *color;      /* NULL = greedy first-fit */
    int32_t A, B, W;
    int32_t mode;
    double t0, t1, pf0, pf1;
    int32_t sweeps;
    uint64_t seed;
    int32_t instance;          /* instance index inside a batch (Philox counter word 2) */
    int32_t replicas;
    int32_t first_sweep;       /* resume support: anneal sweeps [first_sweep, sweeps) */
    int32_t last_sweep;        /* exclusive end; <= 0 means sweeps */
    int32_t check_invariants;  /* recompute G and cut after every window */
    int32_t first_replica;     /* replica index of output row 0 (Philox counter word 3, digest) */
    int32_t stale;             /* 1: every spin of a window decides on the G of the window start
                                  (the stale G of Algorithm 3's parallel threads, Section 5.3)
                                  instead of the running G of R2 */
} oracle_params;

typedef struct {
    int8_t *spins;       /* [replicas * n] original vertex order, in: init if use_init, out: final */
    int32_t use_init;
    int32_t *raw_G;      /* [replicas] G after the last sweep, before repair */
    int32_t *final_G;    /* [replicas] after repair */
    int64_t *raw_cut;    /* [replicas] cut before repair (tracked, checked against recomputation) */
    int64_t *final_cut;  /* [replicas] */
    uint64_t *digest;    /* [replicas * sweeps] or NULL */
    int32_t *G_trace;    /* [replicas * sweeps] or NULL */
    int64_t *cut_trace;  /* [replicas * sweeps] or NULL */
    int64_t invariant_failures;
    int32_t num_colors;
    int32_t do_repair;
    int64_t decision_mismatches; /* flips where "G >= gamma" (the order key) disagreed with the
                                    acceptance test u < thr[clamp(dE)] that decides them; 0 */
} oracle_out;

static int64_t weight_of(const oracle_params *p, int64_t e)
{
    return p->w ? (int64_t)p->w[e] : 1;
}

/* cut_w = sum over undirected edges of w_ij [s_i != s_j]  (Eq. 6 generalised to weights) */
static int64_t cut_of(const oracle_params *p, const int8_t *s_orig)
{
    int64_t c = 0;
    for (int32_t i = 0; i < p->n; ++i)
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
            const int32_t j = p->col[e];
            if (j > i && s_orig[i] != s_orig[j]) c += weight_of(p, e);
        }
    return c;
}

int64_t oracle_cut(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                   const int8_t *spins)
{
    oracle_params p;
    memset(&p, 0, sizeof p);
    p.n = n; p.row_ptr = row_ptr; p.col = col; p.w = w;
    return cut_of(&p, spins);
}

/* H = A (sum s)^2 + B cut_w  (Eq. 4-6) */
int64_t oracle_energy(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                      int32_t A, int32_t B, const int8_t *spins)
{
    int64_t G = 0;
    for (int32_t i = 0; i < n; ++i) G += spins[i];
    return (int64_t)A * G * G + (int64_t)B * oracle_cut(n, row_ptr, col, w, spins);
}

/* Exhaustive minimum over all balanced bisections (|V1| = |V2|, or |G| = 1 for odd n).
 * Vertex 0 is fixed to +1 (the cut is symmetric under a global flip). n <= 26.             */
int oracle_bruteforce_bisection(int32_t n, const int64_t *row_ptr, const int32_t *col,
                                const int32_t *w, int64_t *best_cut, int64_t *num_optimal)
{
    if (n < 2 || n > 26) return ORC_ERR_ARG;
    int8_t *s = (int8_t *)malloc((size_t)n);
    if (!s) return ORC_ERR_OOM;
    int64_t best = INF64, cnt = 0;
    const uint32_t lim = 1u << (n - 1);
    for (uint32_t m = 0; m < lim; ++m) {
        /* vertex 0 -> +1; vertex v>0 -> +1 iff bit v-1 set */
        int32_t G = 1;
        s[0] = 1;
        for (int32_t v = 1; v < n; ++v) {
            s[v] = ((m >> (v - 1)) & 1u) ? 1 : -1;
            G += s[v];
        }
        if (G != 0 && G != 1 && G != -1) continue;
        if ((n % 2 == 0) && G != 0) continue;
        const int64_t c = oracle_cut(n, row_ptr, col, w, s);
        if (c < best) { best = c; cnt = 1; }
        else if (c == best) ++cnt;
    }
    free(s);
    *best_cut = best;
    if (num_optimal) *num_optimal = cnt;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* The annealer (Alg. 3 with readings R1-R5), one instance, all replicas, sequentially.        */
int oracle_anneal(const oracle_params *p, oracle_out *o)
{
    const int32_t n = p->n;
    const int32_t R = p->replicas;
    if (n < 1 || R < 1 || p->A < 0 || p->B < 1 || p->W < 0 || p->sweeps < 1) return ORC_ERR_ARG;
    const int32_t s_begin = p->first_sweep;
    const int32_t s_end = p->last_sweep > 0 ? p->last_sweep : p->sweeps;
    if (s_begin < 0 || s_end > p->sweeps || s_begin > s_end) return ORC_ERR_ARG;
    if (!o->use_init && s_begin != 0) return ORC_ERR_ARG;

    int ecap = oracle_table_ecap(p->mode, p->t0, p->t1, p->pf0, p->pf1, p->sweeps);
    if (ecap < 0) return ecap;
    const int width = 2 * ecap + 1;
    uint64_t *thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)p->sweeps * width);
    int32_t *color = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);   /* orig -> rank */
    int32_t *vert = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);   /* rank -> orig */
    int8_t *s = (int8_t *)malloc((size_t)n);                          /* by rank      */
    int8_t *so = (int8_t *)malloc((size_t)n);                         /* by orig id   */
    int8_t *s0 = (int8_t *)malloc((size_t)n);                         /* window start */
    int64_t *hbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *gbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    uint32_t *ubuf = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n); /* this sweep's draws */
    sort_item *items = (sort_item *)malloc(sizeof(sort_item) * (size_t)n);
    int32_t *cls_lo = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!thr || !color || !rank || !vert || !s || !so || !s0 || !hbuf || !gbuf || !ubuf || !items || !cls_lo) {
        free(thr); free(color); free(rank); free(vert); free(s); free(so); free(s0); free(hbuf);
        free(gbuf); free(ubuf); free(items); free(cls_lo);
        return ORC_ERR_OOM;
    }
    int rc = ORC_OK;
    oracle_build_table(p->mode, p->t0, p->t1, p->pf0, p->pf1, p->sweeps, ecap, thr);

    /* colouring (given or greedy) and its check */
    int32_t ncol;
    if (p->color) {
        ncol = 0;
        for (int32_t v = 0; v < n; ++v) {
            color[v] = p->color[v];
            if (color[v] < 0) { rc = ORC_ERR_COLOR; goto done; }
            if (color[v] + 1 > ncol) ncol = color[v] + 1;
        }
    } else {
        ncol = oracle_greedy_color(n, p->row_ptr, p->col, color);
    }
    for (int32_t v = 0; v < n; ++v)
        for (int64_t e = p->row_ptr[v]; e < p->row_ptr[v + 1]; ++e)
            if (color[p->col[e]] == color[v]) { rc = ORC_ERR_COLOR; goto done; }

    /* rank order: (colour asc, splitmix64(id) asc) -- counting sort by colour, then each class
     * sorted by the hash of the vertex id (R2: a fixed pseudo-random order inside a class) */
    {
        int32_t *cnt = (int32_t *)calloc((size_t)ncol + 1, sizeof(int32_t));
        if (!cnt) { rc = ORC_ERR_OOM; goto done; }
        for (int32_t v = 0; v < n; ++v) cnt[color[v] + 1]++;
        for (int32_t c = 0; c < ncol; ++c) cnt[c + 1] += cnt[c];
        int32_t nclass = 0;
        for (int32_t c = 0; c < ncol; ++c)
            if (cnt[c + 1] > cnt[c]) cls_lo[nclass++] = cnt[c];
        cls_lo[nclass] = n;
        o->num_colors = nclass;
        for (int32_t v = 0; v < n; ++v) vert[cnt[color[v]]++] = v;
        for (int32_t k = 0; k < nclass; ++k) {
            const int32_t lo = cls_lo[k], hi = cls_lo[k + 1];
            hash_item *hi_items = (hash_item *)malloc(sizeof(hash_item) * (size_t)(hi - lo));
            if (!hi_items) { free(cnt); rc = ORC_ERR_OOM; goto done; }
            for (int32_t r = lo; r < hi; ++r) { hi_items[r - lo].key = mix64((uint64_t)vert[r]); hi_items[r - lo].v = vert[r]; }
            qsort(hi_items, (size_t)(hi - lo), sizeof(hash_item), cmp_hash);
            for (int32_t r = lo; r < hi; ++r) vert[r] = hi_items[r - lo].v;
            free(hi_items);
        }
        for (int32_t r = 0; r < n; ++r) rank[vert[r]] = r;
        free(cnt);
    }
    const int32_t nclass = o->num_colors;

    for (int32_t rep = 0; rep < R; ++rep) {
        int8_t *sout = o->spins + (size_t)rep * n;
        /* initial state (Alg. 3 "initialize all s_i"; R4) */
        if (o->use_init) {
            for (int32_t v = 0; v < n; ++v) {
                if (sout[v] != 1 && sout[v] != -1) { rc = ORC_ERR_ARG; goto done; }
                s[rank[v]] = sout[v];
            }
        } else {
            for (int32_t pr = 0; 2 * pr + 1 < n; ++pr) {
                const uint32_t u = draw_word(p->seed, (uint32_t)(pr >> 2), 0xFFFFFFFFu,
                                             (uint32_t)p->instance, (uint32_t)(p->first_replica + rep), pr & 3);
                const int8_t a = (u >> 31) ? -1 : 1;
                s[2 * pr] = a;
                s[2 * pr + 1] = (int8_t)-a;
            }
            if (n % 2) s[n - 1] = -1;
        }
        /* G = sum s (Alg. 3 precompute) and the cut, tracked incrementally from here on */
        int64_t G = 0;
        for (int32_t r = 0; r < n; ++r) G += s[r];
        for (int32_t r = 0; r < n; ++r) so[vert[r]] = s[r];
        int64_t cut = cut_of(p, so);

        for (int32_t sw = s_begin; sw < s_end; ++sw) {
            const uint64_t *row = thr + (size_t)sw * width;
            for (int32_t c = 0; c < nclass; ++c) {
                const int32_t lo = cls_lo[c], hi = cls_lo[c + 1];
                const int32_t Wn = p->W > 0 ? p->W : (hi - lo);
                for (int32_t wlo = lo; wlo < hi; wlo += Wn) {
                    const int32_t whi = (wlo + Wn < hi) ? wlo + Wn : hi;
                    /* local fields (Eq. 2) and thresholds; neighbours lie in other classes */
                    for (int32_t r = wlo; r < whi; ++r) {
                        const int32_t v = vert[r];
                        int64_t h = 0;
                        for (int64_t e = p->row_ptr[v]; e < p->row_ptr[v + 1]; ++e)
                            h += weight_of(p, e) * s[rank[p->col[e]]];
                        hbuf[r] = h;
                        const uint32_t u = draw_word(p->seed, (uint32_t)(r >> 2), (uint32_t)sw,
                                                     (uint32_t)p->instance, (uint32_t)(p->first_replica + rep), r & 3);
                        ubuf[r] = u;
                        const int64_t Es = estar(row, ecap, u);
                        gbuf[r] = (s[r] > 0) ? gamma_plus(h, Es, p->A, p->B)
                                             : gamma_minus(h, Es, p->A, p->B);
                    }
                    /* the two groups of the window, in the canonical order of R2; membership is
                     * the sign at window start, so a spin is decided at most once per sweep */
                    for (int32_t r = wlo; r < whi; ++r) s0[r] = s[r];
                    if (p->stale) {
                        /* stale reading: all spins of the window see the G of the window start,
                         * as threads that read G before any of the window's atomics land */
                        const int64_t Gv = G;
                        for (int32_t r = wlo; r < whi; ++r) {
                            const int64_t dE = (int64_t)p->B * s0[r] * hbuf[r]
                                             + 4 * (int64_t)p->A * (1 - (int64_t)s0[r] * Gv);
                            const int64_t kc = (dE < -ecap ? -ecap : (dE > ecap ? ecap : dE)) + ecap;
                            if ((uint64_t)ubuf[r] < row[kc]) {
                                cut += (int64_t)s[r] * hbuf[r];
                                G -= 2 * (int64_t)s[r];
                                s[r] = (int8_t)-s[r];
                            }
                        }
                    }
                    for (int ph = 0; ph < 2 && !p->stale; ++ph) {
                        const int plus_group = ((sw & 1) == 0) ? (ph == 0) : (ph == 1);
                        int32_t m = 0;
                        for (int32_t r = wlo; r < whi; ++r) {
                            if ((s0[r] > 0) != plus_group) continue;
                            items[m].key = plus_group ? gbuf[r] : -gbuf[r];
                            items[m].rank = r;
                            ++m;
                        }
                        qsort(items, (size_t)m, sizeof(sort_item), cmp_item);
                        for (int32_t t = 0; t < m; ++t) {
                            const int32_t r = items[t].rank;
                            /* the decision itself, from its definition: the energy change of
                             * flipping r at the running G (Eq. 4-6, R1) looked up in this sweep's
                             * row and compared with the draw (Alg. 3's acceptance, R3/R6) */
                            const int64_t dE = (int64_t)p->B * s[r] * hbuf[r]
                                             + 4 * (int64_t)p->A * (1 - (int64_t)s[r] * G);
                            const int64_t kc = (dE < -ecap ? -ecap : (dE > ecap ? ecap : dE)) + ecap;
                            const int flip = (uint64_t)ubuf[r] < row[kc];
                            /* gamma only orders the group (R2); it must say the same */
                            const int by_gamma = plus_group ? (G >= gbuf[r]) : (G <= gbuf[r]);
                            if (flip != by_gamma) o->decision_mismatches++;
                            if (flip) {
                                cut += (int64_t)s[r] * hbuf[r];   /* change of the cut: s_i h_i */
                                G -= 2 * (int64_t)s[r];
                                s[r] = (int8_t)-s[r];
                            }
                        }
                    }
                    if (p->check_invariants) {
                        int64_t g2 = 0;
                        for (int32_t r = 0; r < n; ++r) g2 += s[r];
                        for (int32_t r = 0; r < n; ++r) so[vert[r]] = s[r];
                        if (g2 != G || cut_of(p, so) != cut) o->invariant_failures++;
                    }
                }
            }
            if (o->digest || o->G_trace || o->cut_trace) {
                const size_t idx = (size_t)rep * p->sweeps + sw;
                if (o->digest) {
                    uint64_t d = 0;
                    for (int32_t r = 0; r < n; ++r)
                        if (s[r] > 0) d += digest_term(r, sw, p->first_replica + rep);
                    o->digest[idx] = d;
                }
                if (o->G_trace) o->G_trace[idx] = (int32_t)G;
                if (o->cut_trace) o->cut_trace[idx] = cut;
            }
        }
        o->raw_G[rep] = (int32_t)G;
        o->raw_cut[rep] = cut;

        /* exact-balance repair (R5) */
        const int64_t target = n % 2;
        const int64_t absG = G < 0 ? -G : G;
        if (o->do_repair && absG > target) {
            const int64_t k = (absG - target) / 2;
            const int8_t maj = G > 0 ? 1 : -1;
            int32_t m = 0;
            for (int32_t r = 0; r < n; ++r) {
                if (s[r] != maj) continue;
                const int32_t v = vert[r];
                int64_t h = 0;
                for (int64_t e = p->row_ptr[v]; e < p->row_ptr[v + 1]; ++e)
                    h += weight_of(p, e) * s[rank[p->col[e]]];
                items[m].key = (int64_t)s[r] * h;
                items[m].rank = r;
                ++m;
            }
            qsort(items, (size_t)m, sizeof(sort_item), cmp_item);
            for (int64_t t = 0; t < k; ++t) {
                const int32_t r = items[t].rank;
                s[r] = (int8_t)-s[r];
                G -= 2 * (int64_t)maj;
            }
        }
        for (int32_t r = 0; r < n; ++r) so[vert[r]] = s[r];
        o->final_G[rep] = (int32_t)G;
        o->final_cut[rep] = cut_of(p, so);
        memcpy(sout, so, (size_t)n);
    }
done:
    free(thr); free(color); free(rank); free(vert); free(s); free(so); free(s0); free(hbuf);
    free(gbuf); free(ubuf); free(items); free(cls_lo);
    return rc;
}

/* Sizes of the public structs, so the Python side can check its ctypes layout. */
int oracle_sizeof_params(void) { return (int)sizeof(oracle_params); }
int oracle_sizeof_out(void) { return (int)sizeof(oracle_out); }
