// thin_common.cuh -- point characterisation shared by every lambda-thinning kernel.
//
// The 3x3 test of Sec. 2.1 is a lookup in a 256-entry table indexed by the
// mask of strictly lower neighbours (Gamma^--), ring order E, NE, N, NW, W,
// SW, S, SE = bits 0..7.  The table is generated at compile time from the
// combinatorics of the 8-ring (not from coordinates):
//   * ring positions 0, 2, 4, 6 are the 4-neighbours of x, 1, 3, 5, 7 the corners;
//   * two ring points are 4-adjacent iff their positions are cyclically consecutive;
//   * two ring points are 8-adjacent iff consecutive, or both are 4-neighbours two
//     positions apart (E-N, N-W, W-S, S-E).
// Under the pair (n, nbar) = (8,4):
// T+  = number of 8-components of the neighbours >= F(x)      (Sec. 2.1, n = 8)
// T-- = number of 4-components of the neighbours <  F(x) that hold a 4-neighbour
//       of x                                                   (Sec. 2.1, nbar = 4)
// A second table serves (4,8): T+ counts the 4-components of the neighbours
// >= F(x) that hold a 4-neighbour of x, T-- the 8-components of the lower ones.
#pragma once

#include <cstdint>

namespace thin {

constexpr uint32_t kTabDestructible = 1u << 30;  // T+ == 1 && T-- == 1
constexpr uint32_t kTabDivergent = 1u << 31;     // T-- >= 2
constexpr int kTabLabelShift = 6;                // 3 bits per neighbour: 1 + component, 0 = none

constexpr int uf_root(const int *p, int a)
{
    while (p[a] != a) a = p[a];
    return a;
}

constexpr void uf_join(int *p, int a, int b)
{
    a = uf_root(p, a);
    b = uf_root(p, b);
    if (a != b) p[a] = b;
}

// Table entry for a point whose strictly lower neighbours form `lower`.
constexpr uint32_t point_entry(unsigned lower)
{
    const unsigned upper = ~lower & 0xffu;
    int p[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    for (int i = 0; i < 8; ++i) {
        const int j = (i + 1) & 7;
        if (((upper >> i) & 1u) && ((upper >> j) & 1u)) uf_join(p, i, j);
        const int k = (i + 2) & 7;
        if ((i & 1) == 0 && ((upper >> i) & 1u) && ((upper >> k) & 1u)) uf_join(p, i, k);
    }
    uint32_t tplus = 0;
    for (int i = 0; i < 8; ++i)
        if (((upper >> i) & 1u) && uf_root(p, i) == i) ++tplus;

    uint32_t tminus = 0, labels = 0;
    if ((lower & 0xffu) == 0xffu) {
        tminus = 1;  // one run around the whole ring, it holds 4-neighbours
        for (int i = 0; i < 8; ++i) labels |= 1u << (3 * i);
    } else if (lower & 0xffu) {
        int s = 0;
        while ((lower >> s) & 1u) ++s;  // a position outside Gamma^--
        unsigned run = 0;
        bool has_four = false;
        for (int t = 1; t <= 8; ++t) {
            const int i = (s + t) & 7;
            if ((lower >> i) & 1u) {
                run |= 1u << i;
                if ((i & 1) == 0) has_four = true;
            } else {
                if (run && has_four) {
                    ++tminus;
                    for (int q = 0; q < 8; ++q)
                        if ((run >> q) & 1u) labels |= tminus << (3 * q);
                }
                run = 0;
                has_four = false;
            }
        }
    }
    uint32_t e = tplus | (tminus << 3) | (labels << kTabLabelShift);
    if (tplus == 1 && tminus == 1) e |= kTabDestructible;
    if (tminus >= 2) e |= kTabDivergent;
    return e;
}

// Table entry under (4,8)-adjacency (Sec. 2.1 allows both pairs): T+ counts
// the 4-components of the neighbours >= F(x) that hold a 4-neighbour of x
// (4-adjacent ring points are cyclically consecutive, so these are runs);
// T-- counts the 8-components of the lower neighbours (every ring point is
// 8-adjacent to x), found by union-find over ring 8-adjacency.
constexpr uint32_t point_entry48(unsigned lower)
{
    lower &= 0xffu;
    const unsigned upper = ~lower & 0xffu;
    uint32_t tplus = 0;
    if (upper == 0xffu) {
        tplus = 1;
    } else if (upper) {
        int s = 0;
        while ((upper >> s) & 1u) ++s;  // a position outside Gamma^+
        bool run = false, has_four = false;
        for (int t = 1; t <= 8; ++t) {
            const int i = (s + t) & 7;
            if ((upper >> i) & 1u) {
                run = true;
                if ((i & 1) == 0) has_four = true;
            } else {
                if (run && has_four) ++tplus;
                run = false;
                has_four = false;
            }
        }
    }
    int p[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    for (int i = 0; i < 8; ++i) {
        const int j = (i + 1) & 7;
        if (((lower >> i) & 1u) && ((lower >> j) & 1u)) uf_join(p, i, j);
        const int k = (i + 2) & 7;
        if ((i & 1) == 0 && ((lower >> i) & 1u) && ((lower >> k) & 1u)) uf_join(p, i, k);
    }
    uint32_t tminus = 0, labels = 0;
    int label_of_root[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 8; ++i) {
        if (!((lower >> i) & 1u)) continue;
        const int r = uf_root(p, i);
        if (!label_of_root[r]) label_of_root[r] = int(++tminus);
        labels |= uint32_t(label_of_root[r]) << (3 * i);
    }
    uint32_t e = tplus | (tminus << 3) | (labels << kTabLabelShift);
    if (tplus == 1 && tminus == 1) e |= kTabDestructible;
    if (tminus >= 2) e |= kTabDivergent;
    return e;
}

struct PointTable {
    uint32_t v[256];
};

constexpr PointTable make_point_table(int adj)
{
    PointTable t{};
    for (unsigned m = 0; m < 256; ++m) t.v[m] = adj ? point_entry48(m) : point_entry(m);
    return t;
}

constexpr PointTable kPointTable = make_point_table(0);
constexpr PointTable kPointTable48 = make_point_table(1);

// Shared-memory table block of every kernel: the point table of (8,4), then
// that of (4,8), 256 words each.
constexpr int kTabWords = 512;
constexpr int kTabOffset48 = 256;

#ifdef __CUDACC__

// Lambda rule for a k-divergent point (Sec. 2.1): at least k-1 of the k
// counted lower components c satisfy F(x) - F^-(c) <= lambda, where F^-(c) is
// the largest (rule 0) or smallest (rule 1) value over c.
__device__ __forceinline__ bool divergent_within_lambda(uint32_t e, uint32_t c, const uint32_t nb[8],
                                                        uint32_t lam, int rule)
{
    const uint32_t k = (e >> 3) & 7u;
    const uint32_t init = rule == 0 ? 0u : 0xffffffffu;
    uint32_t f[4] = {init, init, init, init};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t lab = (e >> (kTabLabelShift + 3 * i)) & 7u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (lab == uint32_t(j + 1)) f[j] = rule == 0 ? max(f[j], nb[i]) : min(f[j], nb[i]);
        }
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) cnt += (uint32_t(j) < k && c - f[j] <= lam) ? 1u : 0u;
    return cnt + 1 >= k;
}

// The lowering loop of Sec. 2.2 at one point whose neighbours stay fixed:
// while x may be lowered, F(x) := alpha^-(x, F).  Each step lands on a
// distinct neighbour value, so at most eight steps succeed.  `tab` is the
// point table of the adjacency pair.  mode: bit 0 the F^- reading (0 max,
// 1 min), bit 1 the operator -- 0: lambda-thinning (x is
// lambda-destructible), 1: lambda-skeleton (x is lambda-deletable and not
// lambda-end: lambda-destructible or a peak point, T+ = 0, with
// F(x) - alpha^- <= lambda; and not an end point, one point of Gamma_n^*(x)
// >= F(x), with F(x) - alpha^- > lambda); bit 2 the pair, 0: (8,4), 1: (4,8)
// (n = 4 in the end-point count).  Returns the new value and adds the number
// of steps to `nlow`.
__device__ __forceinline__ uint32_t lower_point(uint32_t c, const uint32_t nb[8], const uint32_t *tab,
                                                uint32_t lam, int mode, int &nlow)
{
    const int rule = mode & 1;
#pragma unroll 1
    for (int it = 0; it < 9; ++it) {
        uint32_t m = 0, alpha = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const bool lt = nb[i] < c;
            m |= (lt ? 1u : 0u) << i;
            alpha = lt ? max(alpha, nb[i]) : alpha;
        }
        if (m == 0) break;
        const uint32_t e = tab[m];
        bool ok = (e & kTabDestructible) != 0;
        if (!ok && (e & kTabDivergent) && lam != 0) ok = divergent_within_lambda(e, c, nb, lam, rule);
        if (mode & 2) {
            const bool shallow = c - alpha <= lam;   // F(x) - alpha^- <= lambda
            const bool peak = (e & 7u) == 0;         // T+ = 0
            const uint32_t near = (mode & 4) ? 0x55u : 0xffu;  // Gamma_n^*(x): 4- or 8-neighbours
            const bool end = __popc(~m & near) == 1;  // one of them in F_k, k = F(x)
            ok = (ok || (peak && shallow)) && !(end && !shallow);
        }
        if (!ok) break;
        c = alpha;
        ++nlow;
    }
    return c;
}

#endif  // __CUDACC__

}  // namespace thin
