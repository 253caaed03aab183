/*
 * CPU oracle for grayscale lambda-thinning under (8,4)-adjacency (and (4,8)).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded restatement
 * of the paper's definitions (Sec. 2.1) and of its lowering loop (Sec. 2.2),
 * run in the fixed 2x2-parity subfield schedule.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it.  The CUDA library
 * never loads it, and the two share no code, header, table or constant.
 *
 * Conventions (an interface, not arithmetic): an image is an int32 array of
 * h rows and w columns, row stride `stride` elements; pixel (x, y) is column
 * x, row y, origin top-left, y growing downwards.  The eight neighbours of a
 * point are listed in ring order E, NE, N, NW, W, SW, S, SE (bit 0..7 of a
 * neighbour mask).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - a section is F_k = {x : F(x) >= k} (Sec. 2.1 prints "F_k >= k");
 *  - a point is simple when T = 1 and Tbar = 1 (Sec. 2.1 prints Tbar = 0,
 *    which would leave only interior points as candidates);
 *  - T-- counts 4-connected components (the complement side of the (8,4)
 *    pair, Sec. 2.1), and only those holding a 4-neighbour of x;
 *  - "components of Gamma^-" in the lambda rule are the components counted
 *    by T--, and F^-(c) is the largest value of F over c (rule R1) or,
 *    selectable, the smallest (rule R2);
 *  - the lowering value is alpha^-(x, F) in every case (Sec. 2.1, 2.2);
 *  - within its phase a point is lowered again and again until it is no
 *    longer lambda-destructible (its neighbours do not move meanwhile);
 *  - border pixels are read as neighbours but never written;
 *  - phases follow parity p = 2 (y & 1) + (x & 1) of the point, in the order
 *    0, 1, 2, 3, 0, ... counted from a global phase index; points of one
 *    parity are pairwise not 8-adjacent, so a phase equals any sequential
 *    order over its points;
 *  - stop after a round of four phases that changed nothing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Gamma_8^*(x) in ring order, as offsets (dx, dy) from x. */
static const int RING_DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
static const int RING_DY[8] = {0, -1, -1, -1, 0, 1, 1, 1};

static int iabs(int a) { return a < 0 ? -a : a; }

/* 4- and 8-adjacency between two points of Z^2, straight from Sec. 2.1:
 * y is 4-adjacent to x if |y1-x1| + |y2-x2| <= 1, 8-adjacent if
 * max(|y1-x1|, |y2-x2|) <= 1; "adjacent" here means distinct points. */
static int adjacent(int n, int ax, int ay, int bx, int by)
{
    int dx = iabs(ax - bx), dy = iabs(ay - by);
    if (dx == 0 && dy == 0) return 0;
    if (n == 4) return dx + dy <= 1;
    return (dx > dy ? dx : dy) <= 1;
}

/*
 * #C_n[x, S]: the number of n-connected components of S (a subset of
 * Gamma_8^*(x), given as a ring bitmask) that hold a point n-adjacent to x
 * (Sec. 2.1).  Found by breadth-first search over the points of S.
 * label[i] receives the index of the counted component holding ring point
 * i, or -1 when i is not in S or its component is not counted.
 */
static int count_components(unsigned S, int n, int label[8])
{
    int comp_of[8];
    int i, ncounted = 0, ncomp = 0;
    int counted_index[8];
    for (i = 0; i < 8; i++) comp_of[i] = -1;
    for (i = 0; i < 8; i++) {
        int queue[8], head = 0, tail = 0, touches_x = 0, j;
        if (!(S & (1u << i)) || comp_of[i] >= 0) continue;
        comp_of[i] = ncomp;
        queue[tail++] = i;
        while (head < tail) {
            int p = queue[head++];
            if (adjacent(n, RING_DX[p], RING_DY[p], 0, 0)) touches_x = 1;
            for (j = 0; j < 8; j++) {
                if ((S & (1u << j)) && comp_of[j] < 0 &&
                    adjacent(n, RING_DX[p], RING_DY[p], RING_DX[j], RING_DY[j])) {
                    comp_of[j] = ncomp;
                    queue[tail++] = j;
                }
            }
        }
        counted_index[ncomp] = touches_x ? ncounted++ : -1;
        ncomp++;
    }
    if (label)
        for (i = 0; i < 8; i++) label[i] = comp_of[i] < 0 ? -1 : counted_index[comp_of[i]];
    return ncounted;
}

/*
 * Connectivity numbers of Sec. 2.1 for a point whose strictly lower
 * neighbours (Gamma^--) form the ring mask `lower`; the neighbours that are
 * greater or equal (Gamma^+) are the rest.  adj 0 is the pair (n, nbar) =
 * (8, 4): n = 8 for sections of F, nbar = 4 for their complements; adj 1 is
 * (4, 8).
 *   T+  = #C_n[x, Gamma^+]        T-- = #C_nbar[x, Gamma^--]
 * label[] gets the T-- component of each neighbour (-1 if none).
 */
int oracle_mask_numbers_adj(int adj, unsigned lower, int *tplus, int *tminus, int label[8])
{
    unsigned plus = (~lower) & 0xffu;
    const int n = adj ? 4 : 8, nbar = adj ? 8 : 4;
    *tplus = count_components(plus, n, 0);
    *tminus = count_components(lower & 0xffu, nbar, label);
    return 0;
}

int oracle_mask_numbers(unsigned lower, int *tplus, int *tminus, int label[8])
{
    return oracle_mask_numbers_adj(0, lower, tplus, tminus, label);
}

/* T++ = #C_8[x, Gamma^++] for the strictly greater neighbours (Sec. 2.1). */
int oracle_tplusplus(unsigned greater)
{
    return count_components(greater & 0xffu, 8, 0);
}

/*
 * Lambda-destructibility of a point of value fx with neighbour values nb[]
 * in ring order (Sec. 2.1):
 *   destructible      <=> x simple for F_k, k = F(x) <=> T+ = 1 and T-- = 1;
 *   k-divergent       <=> T-- = k > 1;
 *   lambda-destructible <=> destructible, or k-divergent with at least k-1
 *   components c of Gamma^-- such that F(x) - F^-(c) <= lambda.
 * rule 0 takes F^-(c) = max of F over c, rule 1 the min.
 * Returns 1 if lambda-destructible and then stores alpha^-(x, F), the
 * largest value over Gamma^-- (Sec. 2.1), in *alpha.
 */
int oracle_lambda_destructible_adj(int adj, const int32_t nb[8], int32_t fx, uint32_t lambda, int rule,
                                   int32_t *alpha)
{
    unsigned lower = 0;
    int i, tplus, tminus, label[8];
    int32_t a = 0;
    int have = 0;
    for (i = 0; i < 8; i++) {
        if (nb[i] < fx) {
            lower |= 1u << i;
            if (!have || nb[i] > a) a = nb[i];
            have = 1;
        }
    }
    if (!lower) return 0; /* Gamma^-- empty: T-- = 0 */
    oracle_mask_numbers_adj(adj, lower, &tplus, &tminus, label);
    if (tplus == 1 && tminus == 1) {
        *alpha = a;
        return 1;
    }
    if (tminus > 1) {
        int c, satisfied = 0;
        for (c = 0; c < tminus; c++) {
            int32_t fm = 0;
            int seen = 0;
            for (i = 0; i < 8; i++) {
                if (label[i] != c) continue;
                if (!seen) fm = nb[i];
                else if (rule == 0 ? nb[i] > fm : nb[i] < fm) fm = nb[i];
                seen = 1;
            }
            if ((int64_t)fx - (int64_t)fm <= (int64_t)lambda) satisfied++;
        }
        if (satisfied >= tminus - 1) {
            *alpha = a;
            return 1;
        }
    }
    return 0;
}

int oracle_lambda_destructible(const int32_t nb[8], int32_t fx, uint32_t lambda, int rule,
                               int32_t *alpha)
{
    return oracle_lambda_destructible_adj(0, nb, fx, lambda, rule, alpha);
}

/*
 * End point for F (Sec. 2.1): x is an end point of the section F_k with
 * k = F(x), i.e. exactly one point of Gamma_n^*(x) lies in F_k (n = 8 for
 * adj 0, n = 4 for adj 1).
 */
static int end_point(int adj, const int32_t nb[8], int32_t fx)
{
    int i, c = 0;
    for (i = 0; i < 8; i++)
        if (adjacent(adj ? 4 : 8, RING_DX[i], RING_DY[i], 0, 0)) c += nb[i] >= fx;
    return c == 1;
}

/*
 * The lambda-skeleton's test (Sec. 2.1, algorithm of Sec. 2.2): x may be
 * lowered when it is lambda-deletable and not lambda-end.
 *   peak point         <=> T+ = 0 (no neighbour >= F(x));
 *   lambda-deletable   <=> lambda-destructible, or a peak point with
 *                          F(x) - alpha^-(x, F) <= lambda;
 *   lambda-end         <=> an end point for F with F(x) - alpha^-(x, F) > lambda.
 * Returns 1 if x may be lowered and then stores alpha^-(x, F) in *alpha.
 */
int oracle_lambda_skeleton_point_adj(int adj, const int32_t nb[8], int32_t fx, uint32_t lambda, int rule,
                                     int32_t *alpha)
{
    unsigned lower = 0;
    int i, tplus, tminus, label[8], deletable, lambda_end;
    int32_t a = 0, tmp;
    int have = 0;
    for (i = 0; i < 8; i++) {
        if (nb[i] < fx) {
            lower |= 1u << i;
            if (!have || nb[i] > a) a = nb[i];
            have = 1;
        }
    }
    if (!lower) return 0; /* alpha^- = F(x): not destructible, not a peak */
    oracle_mask_numbers_adj(adj, lower, &tplus, &tminus, label);
    deletable = oracle_lambda_destructible_adj(adj, nb, fx, lambda, rule, &tmp) ||
                (tplus == 0 && (int64_t)fx - (int64_t)a <= (int64_t)lambda);
    lambda_end = end_point(adj, nb, fx) && (int64_t)fx - (int64_t)a > (int64_t)lambda;
    if (deletable && !lambda_end) {
        *alpha = a;
        return 1;
    }
    return 0;
}

int oracle_lambda_skeleton_point(const int32_t nb[8], int32_t fx, uint32_t lambda, int rule,
                                 int32_t *alpha)
{
    return oracle_lambda_skeleton_point_adj(0, nb, fx, lambda, rule, alpha);
}

/* The test of operator `op` under adjacency pair `adj` (0: (8,4), 1: (4,8)):
 * op 0 = lambda-thinning (lambda-destructible points), op 1 = lambda-skeleton
 * (lambda-deletable, not lambda-end points). */
int oracle_lowerable(int op, int adj, const int32_t nb[8], int32_t fx, uint32_t lambda, int rule, int32_t *alpha)
{
    return op == 1 ? oracle_lambda_skeleton_point_adj(adj, nb, fx, lambda, rule, alpha)
                   : oracle_lambda_destructible_adj(adj, nb, fx, lambda, rule, alpha);
}

static void gather(const int32_t *F, int64_t stride, int x, int y, int32_t nb[8])
{
    int i;
    for (i = 0; i < 8; i++) nb[i] = F[(int64_t)(y + RING_DY[i]) * stride + (x + RING_DX[i])];
}

typedef struct {
    int64_t phases;            /* phases run */
    int64_t rounds;            /* rounds of four phases run, the last one quiet */
    int64_t lowered;           /* lowering steps F(x) := alpha^- performed */
    int64_t last_change_phase; /* global index of the last phase that lowered a point, -1 if none */
    int64_t end_phase;         /* global phase index to resume from */
    int32_t converged;         /* 1 if a quiet round was seen */
} oracle_stats;

/*
 * Sequential lambda-thinning in the subfield schedule (the lowering loop of
 * Sec. 2.2 with the lambda-destructible predicate of Sec. 2.1; op = 1 takes
 * the lambda-skeleton's test instead, see oracle_lowerable).  Rounds of
 * four consecutive phases start at global phase index start_phase; phase g
 * visits, in raster order, the interior points of parity g mod 4 and lowers
 * each one to alpha^- while it stays lambda-destructible.  Stops after a
 * round with no change, or when max_phases phases have run (max_phases < 0:
 * no cap).  F is modified in place.  Returns 0, or 1 if stopped by the cap.
 */
int oracle_thin(int32_t *F, int w, int h, int64_t stride, uint32_t lambda, int rule, int op, int adj,
                int64_t start_phase, int64_t max_phases, oracle_stats *st)
{
    int64_t g = start_phase, run = 0;
    oracle_stats s;
    memset(&s, 0, sizeof s);
    s.last_change_phase = -1;
    for (;;) {
        int r, round_changed = 0;
        for (r = 0; r < 4; r++) {
            int p, x, y, phase_changed = 0;
            if (max_phases >= 0 && run >= max_phases) {
                s.phases = run;
                s.end_phase = g;
                if (st) *st = s;
                return 1;
            }
            p = (int)(((g % 4) + 4) % 4);
            for (y = 1; y < h - 1; y++) {
                for (x = 1; x < w - 1; x++) {
                    int32_t nb[8], alpha;
                    int32_t *fx = &F[(int64_t)y * stride + x];
                    if (2 * (y & 1) + (x & 1) != p) continue;
                    gather(F, stride, x, y, nb);
                    while (oracle_lowerable(op, adj, nb, *fx, lambda, rule, &alpha)) {
                        *fx = alpha;
                        s.lowered++;
                        phase_changed = 1;
                    }
                }
            }
            if (phase_changed) {
                round_changed = 1;
                s.last_change_phase = g;
            }
            g++;
            run++;
        }
        s.rounds++;
        if (!round_changed) break;
    }
    s.phases = run;
    s.end_phase = g;
    s.converged = 1;
    if (st) *st = s;
    return 0;
}

/*
 * Queue-based sequential thinning: a FIFO seeded with every interior point
 * in raster order; pop x, lower it while it is lambda-destructible, and if it
 * moved push those of its eight neighbours that are interior and not already
 * queued (each lowering asks for the neighbours to be re-examined, Sec. 2.2
 * and 3.2; no point is queued twice, Sec. 3.3).  Its result may differ from
 * the subfield schedule; it is compared by invariants only.  Returns the
 * number of lowering steps, or -1 on allocation failure.
 */
int64_t oracle_thin_queue(int32_t *F, int w, int h, int64_t stride, uint32_t lambda, int rule, int op, int adj)
{
    int64_t n = (int64_t)w * h, head = 0, count = 0, lowered = 0;
    int64_t *q;
    unsigned char *inq;
    int x, y, i;
    if (w < 3 || h < 3) return 0;
    q = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    inq = (unsigned char *)calloc((size_t)n, 1);
    if (!q || !inq) {
        free(q);
        free(inq);
        return -1;
    }
    /* circular FIFO of capacity n; a point is in it at most once */
    for (y = 1; y < h - 1; y++)
        for (x = 1; x < w - 1; x++) {
            q[(head + count) % n] = (int64_t)y * w + x;
            count++;
            inq[(int64_t)y * w + x] = 1;
        }
    while (count > 0) {
        int64_t id = q[head];
        int32_t nb[8], alpha, *fx;
        int moved = 0;
        head = (head + 1) % n;
        count--;
        inq[id] = 0;
        x = (int)(id % w);
        y = (int)(id / w);
        fx = &F[(int64_t)y * stride + x];
        gather(F, stride, x, y, nb);
        while (oracle_lowerable(op, adj, nb, *fx, lambda, rule, &alpha)) {
            *fx = alpha;
            lowered++;
            moved = 1;
        }
        if (!moved) continue;
        for (i = 0; i < 8; i++) {
            int nx = x + RING_DX[i], ny = y + RING_DY[i];
            int64_t nid = (int64_t)ny * w + nx;
            if (nx < 1 || ny < 1 || nx > w - 2 || ny > h - 2 || inq[nid]) continue;
            q[(head + count) % n] = nid;
            count++;
            inq[nid] = 1;
        }
    }
    free(q);
    free(inq);
    return lowered;
}

/* Min-heap of (value, raster index) pairs for the minimal-value order. */
typedef struct { int32_t v; int64_t id; } heap_item;

static int heap_less(heap_item a, heap_item b) { return a.v < b.v || (a.v == b.v && a.id < b.id); }

static void heap_push(heap_item *hp, int64_t *n, heap_item it)
{
    int64_t i = (*n)++;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!heap_less(it, hp[par])) break;
        hp[i] = hp[par];
        i = par;
    }
    hp[i] = it;
}

static heap_item heap_pop(heap_item *hp, int64_t *n)
{
    heap_item top = hp[0], last = hp[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && heap_less(hp[c + 1], hp[c])) c++;
        if (!heap_less(hp[c], last)) break;
        hp[i] = hp[c];
        i = c;
    }
    hp[i] = last;
    return top;
}

/*
 * Minimal-value sequential thinning (the selection rule of the algorithm of
 * Sec. 2.2): repeatedly take, among the points the test of `op` accepts, one
 * of minimal value (ties: smallest raster index) and lower it to alpha^-.
 * With op = 1 this is the paper's lambda-skeleton algorithm itself.
 * Candidates sit in a lazy min-heap; a popped entry whose value is stale is
 * dropped, and each lowering re-queues the point and its eight neighbours.
 * Compared with the subfield schedule by invariants only.  Returns the number
 * of lowering steps, or -1 on allocation failure.
 */
int64_t oracle_thin_minvalue(int32_t *F, int w, int h, int64_t stride, uint32_t lambda, int rule, int op, int adj)
{
    int64_t cap, n = 0, lowered = 0;
    heap_item *hp;
    int x, y, i;
    if (w < 3 || h < 3) return 0;
    cap = (int64_t)w * h * 2 + 64;
    hp = (heap_item *)malloc(sizeof(heap_item) * (size_t)cap);
    if (!hp) return -1;
    for (y = 1; y < h - 1; y++)
        for (x = 1; x < w - 1; x++) {
            heap_item it;
            it.v = F[(int64_t)y * stride + x];
            it.id = (int64_t)y * w + x;
            heap_push(hp, &n, it);
        }
    while (n > 0) {
        heap_item it = heap_pop(hp, &n);
        int32_t nb[8], alpha, *fx;
        x = (int)(it.id % w);
        y = (int)(it.id / w);
        fx = &F[(int64_t)y * stride + x];
        if (*fx != it.v) continue; /* stale entry */
        gather(F, stride, x, y, nb);
        if (!oracle_lowerable(op, adj, nb, *fx, lambda, rule, &alpha)) continue;
        *fx = alpha;
        lowered++;
        if (n + 9 > cap) {
            heap_item *nh;
            cap *= 2;
            nh = (heap_item *)realloc(hp, sizeof(heap_item) * (size_t)cap);
            if (!nh) {
                free(hp);
                return -1;
            }
            hp = nh;
        }
        it.v = *fx;
        heap_push(hp, &n, it);
        for (i = 0; i < 8; i++) {
            int nx = x + RING_DX[i], ny = y + RING_DY[i];
            heap_item nt;
            if (nx < 1 || ny < 1 || nx > w - 2 || ny > h - 2) continue;
            nt.id = (int64_t)ny * w + nx;
            nt.v = F[(int64_t)ny * stride + nx];
            heap_push(hp, &n, nt);
        }
    }
    free(hp);
    return lowered;
}

/* Number of interior points the test of `op` accepts for F (0 at a fixed point). */
int64_t oracle_count_lambda_destructible(const int32_t *F, int w, int h, int64_t stride,
                                         uint32_t lambda, int rule, int op, int adj)
{
    int64_t c = 0;
    int x, y;
    for (y = 1; y < h - 1; y++)
        for (x = 1; x < w - 1; x++) {
            int32_t nb[8], alpha;
            gather(F, stride, x, y, nb);
            if (oracle_lowerable(op, adj, nb, F[(int64_t)y * stride + x], lambda, rule, &alpha)) c++;
        }
    return c;
}

/*
 * Number of n-connected components (n = 8 or 4) of the section
 * X = {p : F(p) >= k} (complement = 0) or of its complement {p : F(p) < k}
 * (complement = 1), on the finite w x h grid, by breadth-first search.
 * `skip_x, skip_y`: one point whose membership is flipped (-1 for none), so
 * that X \ {x} or Xbar U {x} can be counted without copying F.
 * Returns -1 on allocation failure.
 */
int64_t oracle_count_section_components(const int32_t *F, int w, int h, int64_t stride, int32_t k,
                                        int n, int complement, int flip_x, int flip_y)
{
    int64_t N = (int64_t)w * h, comps = 0, id;
    int32_t *queue;
    unsigned char *seen;
    if (N == 0) return 0;
    queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    seen = (unsigned char *)calloc((size_t)N, 1);
    if (!queue || !seen) {
        free(queue);
        free(seen);
        return -1;
    }
#define IN_SET(px, py)                                                                  \
    ((((F[(int64_t)(py) * stride + (px)] >= k) ^ (complement != 0)) ^                   \
      ((px) == flip_x && (py) == flip_y)))
    for (id = 0; id < N; id++) {
        int x0 = (int)(id % w), y0 = (int)(id / w);
        int64_t head = 0, tail = 0;
        if (seen[id] || !IN_SET(x0, y0)) continue;
        comps++;
        seen[id] = 1;
        queue[tail++] = (int32_t)id;
        while (head < tail) {
            int32_t cur = queue[head++];
            int cx = cur % w, cy = cur / w, dx, dy;
            for (dy = -1; dy <= 1; dy++)
                for (dx = -1; dx <= 1; dx++) {
                    int nx = cx + dx, ny = cy + dy;
                    int64_t nid;
                    if (nx < 0 || ny < 0 || nx >= w || ny >= h) continue;
                    if (!adjacent(n, cx, cy, nx, ny)) continue;
                    nid = (int64_t)ny * w + nx;
                    if (seen[nid] || !IN_SET(nx, ny)) continue;
                    seen[nid] = 1;
                    queue[tail++] = (int32_t)nid;
                }
        }
    }
#undef IN_SET
    free(queue);
    free(seen);
    return comps;
}

/*
 * Brute-force global destructibility of the point (x, y): with k = F(x),
 * removing x from F_k keeps the number of n-components of F_k and the number
 * of nbar-components of its complement (a simple point changes neither,
 * Sec. 2.1); (n, nbar) = (8, 4) for adj 0, (4, 8) for adj 1.  Returns 1 if
 * both counts are kept, 0 if not, -1 on error.
 */
int oracle_global_destructible_adj(int adj, const int32_t *F, int w, int h, int64_t stride, int x, int y)
{
    int32_t k = F[(int64_t)y * stride + x];
    const int n = adj ? 4 : 8, nbar = adj ? 8 : 4;
    int64_t a = oracle_count_section_components(F, w, h, stride, k, n, 0, -1, -1);
    int64_t b = oracle_count_section_components(F, w, h, stride, k, n, 0, x, y);
    int64_t c = oracle_count_section_components(F, w, h, stride, k, nbar, 1, -1, -1);
    int64_t d = oracle_count_section_components(F, w, h, stride, k, nbar, 1, x, y);
    if (a < 0 || b < 0 || c < 0 || d < 0) return -1;
    return a == b && c == d;
}

int oracle_global_destructible(const int32_t *F, int w, int h, int64_t stride, int x, int y)
{
    return oracle_global_destructible_adj(0, F, w, h, stride, x, y);
}
