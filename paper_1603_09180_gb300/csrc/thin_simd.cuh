// thin_simd.cuh -- the point test of Sec. 2.1 and the lowering loop of
// Sec. 2.2 on four points of one parity at once, shared by the engines.
//
// A work item is the four points (x0 + px + 2k, y), k = 0..3, of one parity in
// an 8-pixel aligned block of row y.  The callers pass pointers to that block
// in rows y - 1, y and y + 1 (any of them may live in another block's shared
// memory); the rows must hold readable pixels from 1 pixel left to 1 pixel
// right of the block (u8: the aligned words just left and right of it).
#pragma once

#include <cstdint>

#include "thin_common.cuh"

namespace thin {

constexpr uint32_t kMsb8 = 0x80808080u;
constexpr uint32_t kLsb8 = 0x01010101u;

// Four unsigned byte comparisons a < b at once: bit 7 of each byte of the
// result is set where byte(a) < byte(b); all other bits are 0.
// bl = b & 0x7f7f7f7f, bh = b & 0x80808080.  The subtraction of the low
// seven bits cannot borrow across bytes; bit 7 is then fixed up by hand.
__device__ __forceinline__ uint32_t lt8(uint32_t a, uint32_t b, uint32_t bl, uint32_t bh)
{
    const uint32_t x = a ^ b;
    const uint32_t r = (a | kMsb8) - bl;
    const uint32_t dh = (r ^ ~x) & kMsb8;  // bit 7 of the true byte difference a - b
    return (x & bh) | (~x & dh);           // borrow out of the byte
}

// 0xff in each byte whose bit 7 is set, else 0x00 (prmt sign replication).
__device__ __forceinline__ uint32_t msb_to_mask(uint32_t v)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xba98;" : "=r"(r) : "r"(v));
    return r;
}

// Rotations of each byte seen as the 8-ring of neighbour bits:
// rot_prev puts bit i-1 at bit i, rot_next puts bit i+1 at bit i.
__device__ __forceinline__ uint32_t rot_prev(uint32_t v) { return ((v << 1) & 0xfefefefeu) | ((v >> 7) & kLsb8); }
__device__ __forceinline__ uint32_t rot_next(uint32_t v) { return ((v >> 1) & 0x7f7f7f7fu) | ((v << 7) & kMsb8); }

// Bit 7 set in every nonzero byte.
__device__ __forceinline__ uint32_t nonzero8(uint32_t v) { return (((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v) & kMsb8; }

// Merge eight per-direction comparison results (bit 7 per byte) into the
// ring mask of each point (byte k = mask of point k, bit d = direction d).
__device__ __forceinline__ uint32_t merge_dirs(const uint32_t lt[8])
{
    return (lt[0] >> 7) | (lt[1] >> 6) | (lt[2] >> 5) | (lt[3] >> 4) | (lt[4] >> 3) | (lt[5] >> 2) |
           (lt[6] >> 1) | lt[7];
}

// Lambda-destructibility (Sec. 2.1) of four points of one parity at once
// (bytes of `c`), neighbours nb[d] in ring order E, NE, N, NW, W, SW, S, SE.
// For each point: Gamma^-- is its lower-neighbour mask (byte of M); T-- is the
// number of runs of M once isolated lower corners (those with no lower
// 4-neighbour beside them, never 4-adjacent to x) are dropped; under (8,4),
// T+ = T-- except when no 4-neighbour is lower (T-- = 0) or all eight are
// (T+ = 0), so "destructible" is "exactly one run start".  k-divergent points
// (two or more runs) are lambda-destructible when at most one of their
// counted components fails F(x) - F^-(c) <= lambda.  mode: bit 0 the F^-
// reading (0 max, 1 min); bit 1 set asks for the lambda-skeleton's test
// instead (lambda-deletable and not lambda-end, Sec. 2.1-2.2): a peak point
// (all eight lower, T+ = 0) also qualifies when F(x) - alpha^- <= lambda, and
// an end point (exactly one neighbour >= F(x)) is kept when
// F(x) - alpha^- > lambda.  Returns 0x01 in the bytes of the points that may
// be lowered, among those set in `vm`.
// Lower-neighbour masks of the four points at centre values c (byte k = mask of point k).
__device__ __forceinline__ uint32_t lower_mask4(uint32_t c, const uint32_t nb[8])
{
    const uint32_t bl = c & 0x7f7f7f7fu, bh = c & kMsb8;
    uint32_t lt[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) lt[d] = lt8(nb[d], c, bl, bh);
    return merge_dirs(lt);
}

// Byte-wise arithmetic through 16-bit lanes.  The 16-bit lane minimum and
// maximum are single instructions; their 4-byte forms are not (measured on
// the GB300: __vmaxu4 and __vsubus4 cost about seven times __vmaxu2).  A word's
// even bytes (mask 0x00ff00ff) and odd bytes (0xff00ff00), each left in
// place, are two pairs of 16-bit lanes whose order is the bytes' order.
constexpr uint32_t kEven8 = 0x00ff00ffu, kOdd8 = 0xff00ff00u;

// c - l per byte, floored at 0.
__device__ __forceinline__ uint32_t subus8(uint32_t c, uint32_t l)
{
    const uint32_t ce = c & kEven8, co = c & kOdd8;
    return (ce - __vminu2(ce, l & kEven8)) | (co - __vminu2(co, l & kOdd8));
}

// c + l per byte, capped at 255: c + min(l, 255 - c), which stays in the lane.
__device__ __forceinline__ uint32_t addus8(uint32_t c, uint32_t l)
{
    return ((c & kEven8) + __vminu2(l & kEven8, ~c & kEven8)) | ((c & kOdd8) + __vminu2(l & kOdd8, ~c & kOdd8));
}

// alpha^- of the four points given their lower masks M: the largest lower
// neighbour, by trees of maxima over the even and the odd bytes (0 where a
// mask is empty).
__device__ __forceinline__ uint32_t alpha4(const uint32_t nb[8], uint32_t M)
{
    uint32_t e[8], o[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const uint32_t v = nb[d] & (((M >> d) & kLsb8) * 0xffu);
        e[d] = v & kEven8;
        o[d] = v & kOdd8;
    }
    const uint32_t me = __vmaxu2(__vmaxu2(__vmaxu2(e[0], e[1]), __vmaxu2(e[2], e[3])),
                                 __vmaxu2(__vmaxu2(e[4], e[5]), __vmaxu2(e[6], e[7])));
    const uint32_t mo = __vmaxu2(__vmaxu2(__vmaxu2(o[0], o[1]), __vmaxu2(o[2], o[3])),
                                 __vmaxu2(__vmaxu2(o[4], o[5]), __vmaxu2(o[6], o[7])));
    return me | mo;
}

// Bit 7 set in each byte where a and b are equal.
__device__ __forceinline__ uint32_t eq8(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;
    return ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & kMsb8;
}

// Masks of the neighbours equal to the centre values c (byte k = mask of point k).
// A point just lowered to c = alpha^- loses exactly these from its lower mask:
// every other lower neighbour is below alpha^-, every other neighbour above c.
__device__ __forceinline__ uint32_t equal_mask4(uint32_t c, const uint32_t nb[8])
{
    uint32_t e[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) e[d] = eq8(nb[d], c);
    return merge_dirs(e);
}

// FIX >= 0 fixes the mode word at compile time (the kernels pass the common
// mode, lambda-thinning with F^- = max, this way); FIX < 0 reads `mode`.
template <int FIX = -1>
__device__ __forceinline__ uint32_t decide4m(uint32_t c, const uint32_t nb[8], uint32_t vm, uint32_t lam, int mode, uint32_t M);

template <int FIX = -1>
__device__ __forceinline__ uint32_t decide4(uint32_t c, const uint32_t nb[8], uint32_t vm, uint32_t lam, int mode, uint32_t &M)
{
    M = lower_mask4(c, nb);
    return decide4m<FIX>(c, nb, vm, lam, mode, M);
}

// The decision of Sec. 2.1 from masks alone (bit d of byte k: direction d of
// point k): M the lower neighbours, and below() the neighbours below
// F(x) - lambda (none when F(x) <= lambda), computed only when the lambda rule
// or the skeleton's test needs it.  The test depends on the pixel values
// through these two masks only.
template <int FIX, typename Below>
__device__ __forceinline__ uint32_t decide_masks(uint32_t M, uint32_t vm, uint32_t lam, int mode_rt, Below below)
{
    const int mode = FIX >= 0 ? FIX : mode_rt;
    const int rule = mode & 1;
    const uint32_t iso = M & 0xaaaaaaaau & ~rot_prev(M) & ~rot_next(M);
    const uint32_t mc = M ^ iso;                              // counted lower neighbours
    const uint32_t st = mc & ~rot_prev(mc);                   // starts of their runs
    const uint32_t t = st & ((st | kMsb8) - kLsb8);           // starts minus the lowest one
    const uint32_t nzt = nonzero8(t);
    uint32_t ok = ((nonzero8(st) & ~nzt) >> 7) & vm;          // destructible
    const uint32_t dv = (nzt >> 7) & vm;                      // k-divergent
    uint32_t D = 0;
    bool haveD = false;
    if (lam != 0 && dv) {
        D = below();
        haveD = true;
        const uint32_t deep = D & mc;
        // The counted components are the cyclic runs of mc.  F^- = max: a component fails when no
        // member is shallow (value >= F(x) - lambda); F^- = min: when some member is deep.  The
        // probe bits are carried towards the start of their run (a run of a k-divergent point has
        // at most 5 bits), so a run's start is reached exactly when the run holds a probe bit.
        const uint32_t probe = rule == 0 ? (mc & ~deep) : deep;
        uint32_t fill = probe;
#pragma unroll
        for (int i = 0; i < 4; ++i) fill |= rot_next(fill) & mc;
        const uint32_t bad = rule == 0 ? (st & ~fill) : (st & fill);  // failing components, by their start
        const uint32_t two = nonzero8(bad & ((bad | kMsb8) - kLsb8));   // two or more of them
        ok |= (~two >> 7) & dv;
    }
    if (mode & 2) {
        // shallow: some lower neighbour >= F(x) - lambda, i.e. F(x) - alpha^- <= lambda
        if (!haveD) D = below();
        const uint32_t shallow = nonzero8(M & ~D);
        const uint32_t U = ~M;                                   // neighbours >= F(x), per byte
        const uint32_t peak = ~nonzero8(U) & kMsb8;              // none: T+ = 0
        const uint32_t end = nonzero8(U) & ~nonzero8(U & ((U | kMsb8) - kLsb8));  // exactly one
        ok = (ok | ((peak & shallow) >> 7)) & ~((end & ~shallow) >> 7) & vm;
    }
    return ok & 0x01010101u;
}

// decide4 with the lower masks M of the centre values c already computed.
template <int FIX>
__device__ __forceinline__ uint32_t decide4m(uint32_t c, const uint32_t nb[8], uint32_t vm, uint32_t lam, int mode_rt, uint32_t M)
{
    return decide_masks<FIX>(M, vm, lam, mode_rt, [&] {
        const uint32_t lrep = (lam > 255u ? 255u : lam) * kLsb8;
        const uint32_t cl = subus8(c, lrep);
        const uint32_t cll = cl & 0x7f7f7f7fu, clh = cl & kMsb8;
        uint32_t dp[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) dp[d] = lt8(nb[d], cl, cll, clh);
        return merge_dirs(dp);
    });
}

// Which neighbours of a lowered point must be tested again.  The test of a
// neighbour q sees the point only through two bits: is it below F(q), and is
// it below F(q) - lambda.  The point went from c0 down to c1, and no neighbour
// lies strictly between two successive values of its lowering loop (each step
// goes to the largest lower neighbour), so neither bit can change for a
// neighbour q with F(q) <= c1 (the point stays >= F(q)), nor, for lambda-thinning,
// with F(q) > c0 + lambda (the point was already below F(q) - lambda).  The
// other neighbours are marked: byte k of the result holds the ring directions
// of point k to mark (MARK 1: F(q) > c1; MARK 2: also F(q) <= c0 + lambda
// where `cap` is set: the bound costs a compare per direction, which saves
// more tests than it costs in a batch but not in the wide mode's tail).
// Mlast: per moved point, its lower-neighbour mask before its last lowering
// step, which is {F(q) <= c1}.  The decision of Sec. 2.1 depends on the
// neighbour values only through those two masks, in both operators.
template <int MARK>
__device__ __forceinline__ uint32_t marks8(uint32_t okacc, uint32_t Mlast, uint32_t c0, const uint32_t nb[8], uint32_t lam,
                                           bool cap)
{
    uint32_t aff = ~Mlast & (okacc * 0xffu);
    if (MARK == 2 && cap && aff) {
        const uint32_t t = addus8(c0, (lam > 255u ? 255u : lam) * kLsb8);  // c0 + lambda, saturated
        uint32_t gt[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) gt[d] = lt8(t, nb[d], nb[d] & 0x7f7f7f7fu, nb[d] & kMsb8);
        aff &= ~merge_dirs(gt);
    }
    return aff;
}

// The lowering loop of Sec. 2.2 on the four points: while a point is
// lambda-destructible, F(x) := alpha^-(x, F), its neighbours fixed.  Returns
// the bytes lowered (0x01 each) over all iterations; `c` receives the new
// values, `nin` the lowering steps of the points also in `in`, `aff` the
// neighbours to test again (marks8; every neighbour of a moved point when
// MARK is 0).
template <int FIX = -1, int MARK = 0>
__device__ __forceinline__ uint32_t lower4(uint32_t &c, const uint32_t nb[8], uint32_t vm, uint32_t in,
                                           uint32_t lam, int mode, int &nin, uint32_t &aff, bool cap = true)
{
    uint32_t okacc = 0, Mlast = 0;
    const uint32_t c0 = c;
    uint32_t M = lower_mask4(c, nb);
#pragma unroll 1
    for (int it = 0; it < 9; ++it) {
        const uint32_t ok = decide4m<FIX>(c, nb, vm, lam, mode, M);
        if (!ok) break;
        const uint32_t alpha = alpha4(nb, M);
        const uint32_t okm = ok * 0xffu;
        c = (alpha & okm) | (c & ~okm);
        if (MARK) Mlast = (M & okm) | (Mlast & ~okm);
        okacc |= ok;
        nin += __popc(ok & in);
        M &= ~equal_mask4(c, nb);  // unmoved points: no neighbour equal to c is lower
    }
    aff = MARK ? marks8<MARK>(okacc, Mlast, c0, nb, lam, cap) : okacc * 0xffu;
    return okacc;
}

// lower4 for points whose first test already ran: `ok` holds its result
// (0x01 per byte that may be lowered at the current values).
template <int FIX = -1, int MARK = 0>
__device__ __forceinline__ uint32_t lower4_tested(uint32_t &c, const uint32_t nb[8], uint32_t vm, uint32_t in,
                                                  uint32_t ok, uint32_t lam, int mode, int &nin, uint32_t &aff,
                                                  bool cap = true)
{
    uint32_t okacc = 0, Mlast = 0;
    const uint32_t c0 = c;
    uint32_t M = lower_mask4(c, nb);
#pragma unroll 1
    for (int it = 0; it < 9; ++it) {
        if (!ok) break;
        const uint32_t alpha = alpha4(nb, M);
        const uint32_t okm = ok * 0xffu;
        c = (alpha & okm) | (c & ~okm);
        if (MARK) Mlast = (M & okm) | (Mlast & ~okm);
        okacc |= ok;
        nin += __popc(ok & in);
        M &= ~equal_mask4(c, nb);
        ok = decide4m<FIX>(c, nb, vm, lam, mode, M);
    }
    aff = MARK ? marks8<MARK>(okacc, Mlast, c0, nb, lam, cap) : okacc * 0xffu;
    return okacc;
}

// Gathers a u8 work item: the centre bytes and the eight neighbour vectors of
// the four points.  ra, rb, rc point at the 8-byte aligned block in rows y - 1,
// y, y + 1; the words at -4 and +8 of each must be readable.  `other` gets the
// bytes of row y of the other column parity (to rebuild the block).
__device__ __forceinline__ void gather_u8(const uint8_t *ra, const uint8_t *rb, const uint8_t *rc, int px,
                                          uint32_t nb[8], uint32_t &c, uint32_t &other)
{
    const uint2 wa = *reinterpret_cast<const uint2 *>(ra);
    const uint2 wb = *reinterpret_cast<const uint2 *>(rb);
    const uint2 wc = *reinterpret_cast<const uint2 *>(rc);
    const uint32_t Ea = __byte_perm(wa.x, wa.y, 0x6420), Oa = __byte_perm(wa.x, wa.y, 0x7531);
    const uint32_t Eb = __byte_perm(wb.x, wb.y, 0x6420), Ob = __byte_perm(wb.x, wb.y, 0x7531);
    const uint32_t Ec = __byte_perm(wc.x, wc.y, 0x6420), Oc = __byte_perm(wc.x, wc.y, 0x7531);
    if (px == 0) {
        const uint32_t La = *reinterpret_cast<const uint32_t *>(ra - 4);
        const uint32_t Lb = *reinterpret_cast<const uint32_t *>(rb - 4);
        const uint32_t Lc = *reinterpret_cast<const uint32_t *>(rc - 4);
        c = Eb;
        other = Ob;
        nb[0] = Ob;
        nb[1] = Oa;
        nb[2] = Ea;
        nb[3] = __byte_perm(La, Oa, 0x6543);
        nb[4] = __byte_perm(Lb, Ob, 0x6543);
        nb[5] = __byte_perm(Lc, Oc, 0x6543);
        nb[6] = Ec;
        nb[7] = Oc;
    } else {
        const uint32_t Ra = *reinterpret_cast<const uint32_t *>(ra + 8);
        const uint32_t Rb = *reinterpret_cast<const uint32_t *>(rb + 8);
        const uint32_t Rc = *reinterpret_cast<const uint32_t *>(rc + 8);
        c = Ob;
        other = Eb;
        nb[0] = __byte_perm(Eb, Rb, 0x4321);
        nb[1] = __byte_perm(Ea, Ra, 0x4321);
        nb[2] = Oa;
        nb[3] = Ea;
        nb[4] = Eb;
        nb[5] = Ec;
        nb[6] = Oc;
        nb[7] = __byte_perm(Ec, Rc, 0x4321);
    }
}

// One u8 work item, tested only: 0x01 in the bytes of the points that would be lowered now.
template <int FIX = -1>
__device__ __forceinline__ uint32_t test_u8(const uint8_t *ra, const uint8_t *rb, const uint8_t *rc, int px,
                                            uint32_t vm, uint32_t lam, int mode)
{
    uint32_t nb[8], c, other, M;
    gather_u8(ra, rb, rc, px, nb, c, other);
    return decide4<FIX>(c, nb, vm, lam, mode, M);
}

// One u8 work item, lowered: the lowering loop on its four points, the block written back.
// aff: the neighbours to test again (lower4).
template <int FIX = -1, int MARK = 0>
__device__ __forceinline__ uint32_t item_u8(const uint8_t *ra, uint8_t *rb, const uint8_t *rc, int px, uint32_t vm,
                                            uint32_t in, uint32_t lam, int mode, int &nin, uint32_t &aff, bool cap = true)
{
    uint32_t nb[8], c, other;
    gather_u8(ra, rb, rc, px, nb, c, other);
    const uint32_t moved = lower4<FIX, MARK>(c, nb, vm, in, lam, mode, nin, aff, cap);
    if (moved) {
        uint2 out;
        if (px == 0)
            out = make_uint2(__byte_perm(c, other, 0x5140), __byte_perm(c, other, 0x7362));
        else
            out = make_uint2(__byte_perm(other, c, 0x5140), __byte_perm(other, c, 0x7362));
        *reinterpret_cast<uint2 *>(rb) = out;
    }
    return moved;
}

// item_u8 for a work item whose first test already ran (result `ok`).
template <int FIX = -1, int MARK = 0>
__device__ __forceinline__ uint32_t item_u8_tested(const uint8_t *ra, uint8_t *rb, const uint8_t *rc, int px,
                                                   uint32_t vm, uint32_t in, uint32_t ok, uint32_t lam, int mode, int &nin,
                                                   uint32_t &aff, bool cap = true)
{
    uint32_t nb[8], c, other;
    gather_u8(ra, rb, rc, px, nb, c, other);
    const uint32_t moved = lower4_tested<FIX, MARK>(c, nb, vm, in, ok, lam, mode, nin, aff, cap);
    if (moved) {
        uint2 out;
        if (px == 0)
            out = make_uint2(__byte_perm(c, other, 0x5140), __byte_perm(c, other, 0x7362));
        else
            out = make_uint2(__byte_perm(other, c, 0x5140), __byte_perm(other, c, 0x7362));
        *reinterpret_cast<uint2 *>(rb) = out;
    }
    return moved;
}

// One work item through the point table (u16 images, and u8 images under
// (4,8)): the same four points, one at a time.  ra, rb, rc point at the
// block's first pixel in rows y - 1, y, y + 1; `tab` is the point table of
// the adjacency pair in mode bit 2.
template <typename T>
__device__ __forceinline__ uint32_t item_table(const T *ra, T *rb, const T *rc, int px, uint32_t vm, uint32_t in,
                                               const uint32_t *tab, uint32_t lam, int mode, int &nin)
{
    uint32_t moved = 0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        if (!((vm >> (8 * k)) & 1u)) continue;
        const int x = px + 2 * k;
        uint32_t nb[8] = {rb[x + 1], ra[x + 1], ra[x], ra[x - 1], rb[x - 1], rc[x - 1], rc[x], rc[x + 1]};
        int nl = 0;
        const uint32_t c2 = lower_point(rb[x], nb, tab, lam, mode, nl);
        if (nl) {
            rb[x] = static_cast<T>(c2);
            moved |= 1u << (8 * k);
            if ((in >> (8 * k)) & 1u) nin += nl;
        }
    }
    return moved;
}

// ---------------------------------------------------------------------------
// u16 images under (8,4): the same four points, two per 32-bit word in 16-bit
// lanes (word A holds points 0 and 1, word B points 2 and 3).  The pixel
// comparisons run per lane; their results are brought to the byte-per-point
// mask format, and the decision is decide_masks, as for u8.

constexpr uint32_t kMsb16 = 0x80008000u;

// Two unsigned 16-bit comparisons a < b at once: bit 15 of each lane set where
// lane(a) < lane(b) (the borrow trick of lt8 on 16-bit lanes).
__device__ __forceinline__ uint32_t lt16(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;
    const uint32_t r = (a | kMsb16) - (b & 0x7fff7fffu);
    const uint32_t dh = (r ^ ~x) & kMsb16;
    return (x & b & kMsb16) | (~x & dh);
}

// Bit 15 of each lane set where the lanes of a and b are equal.
__device__ __forceinline__ uint32_t eq16(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;
    return ~(((x & 0x7fff7fffu) + 0x7fff7fffu) | x) & kMsb16;
}

// Lane results of words A and B (bit 15 per lane) as bit 7 of bytes 0..3.
__device__ __forceinline__ uint32_t lanes_to_bytes(uint32_t a, uint32_t b)
{
    return __byte_perm(a, b, 0x7531) & kMsb8;
}

struct Px16 {
    uint32_t nbA[8], nbB[8];  // neighbours in ring order, per word
    uint32_t cA, cB;          // centre values
};

// Masks of the neighbours below the centre values (byte k = point k).
__device__ __forceinline__ uint32_t lower_mask16(const Px16 &P, uint32_t cA, uint32_t cB)
{
    uint32_t lt[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) lt[d] = lanes_to_bytes(lt16(P.nbA[d], cA), lt16(P.nbB[d], cB));
    return merge_dirs(lt);
}

__device__ __forceinline__ uint32_t equal_mask16(const Px16 &P)
{
    uint32_t e[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) e[d] = lanes_to_bytes(eq16(P.nbA[d], P.cA), eq16(P.nbB[d], P.cB));
    return merge_dirs(e);
}

// Per-lane masks (0xffff) of the points whose byte in m is 0x01.
__device__ __forceinline__ uint32_t lanes_of_bytes_lo(uint32_t m) { return __byte_perm(m, 0, 0x1100) * 0xffu; }
__device__ __forceinline__ uint32_t lanes_of_bytes_hi(uint32_t m) { return __byte_perm(m, 0, 0x3322) * 0xffu; }

// alpha^- of the four points: the largest lower neighbour, per lane.
__device__ __forceinline__ void alpha16(const Px16 &P, uint32_t M, uint32_t &aA, uint32_t &aB)
{
    aA = 0;
    aB = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const uint32_t t = (M >> d) & kLsb8;
        aA = __vmaxu2(aA, P.nbA[d] & lanes_of_bytes_lo(t));
        aB = __vmaxu2(aB, P.nbB[d] & lanes_of_bytes_hi(t));
    }
}

template <int FIX>
__device__ __forceinline__ uint32_t decide16m(const Px16 &P, uint32_t vm, uint32_t lam, int mode,
                                              uint32_t M)
{
    return decide_masks<FIX>(M, vm, lam, mode, [&] {
        const uint32_t lrep = (lam > 65535u ? 65535u : lam) * 0x00010001u;
        // c - lambda per lane, floored at 0
        return lower_mask16(P, P.cA - __vminu2(P.cA, lrep), P.cB - __vminu2(P.cB, lrep));
    });
}

// marks8 for u16 items (c0A, c0B: the values before the lowering loop).
template <int MARK>
__device__ __forceinline__ uint32_t marks16(const Px16 &P, uint32_t okacc, uint32_t Mlast, uint32_t c0A, uint32_t c0B,
                                            uint32_t lam, bool cap)
{
    uint32_t aff = ~Mlast & (okacc * 0xffu);
    if (MARK == 2 && cap && aff) {
        const uint32_t lrep = (lam > 65535u ? 65535u : lam) * 0x00010001u;
        // c0 + lambda per lane, capped at 65535: c0 + min(lambda, 65535 - c0)
        const uint32_t tA = c0A + __vminu2(lrep, ~c0A), tB = c0B + __vminu2(lrep, ~c0B);
        uint32_t gt[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) gt[d] = lanes_to_bytes(lt16(tA, P.nbA[d]), lt16(tB, P.nbB[d]));
        aff &= ~merge_dirs(gt);
    }
    return aff;
}

// The lowering loop on the four points (u16).  ok: the result of a first test
// already made at the current values, or ~0u to test first.  Returns the bytes
// lowered (0x01 each); P.cA, P.cB receive the new values, aff the neighbours
// to test again (marks16; every neighbour of a moved point when MARK is 0).
template <int FIX, int MARK = 0>
__device__ __forceinline__ uint32_t lower16(Px16 &P, uint32_t vm, uint32_t in, uint32_t ok, uint32_t lam, int mode, int &nin,
                                            uint32_t &aff, bool cap = true)
{
    uint32_t okacc = 0, Mlast = 0;
    const uint32_t c0A = P.cA, c0B = P.cB;
    uint32_t M = lower_mask16(P, P.cA, P.cB);
    if (ok == ~0u) ok = decide16m<FIX>(P, vm, lam, mode, M);
#pragma unroll 1
    for (int it = 0; it < 9; ++it) {
        if (!ok) break;
        uint32_t aA, aB;
        alpha16(P, M, aA, aB);
        const uint32_t mA = lanes_of_bytes_lo(ok), mB = lanes_of_bytes_hi(ok);
        P.cA = (aA & mA) | (P.cA & ~mA);
        P.cB = (aB & mB) | (P.cB & ~mB);
        if (MARK) {
            const uint32_t okm = ok * 0xffu;
            Mlast = (M & okm) | (Mlast & ~okm);
        }
        okacc |= ok;
        nin += __popc(ok & in);
        M &= ~equal_mask16(P);  // unmoved points: no neighbour equal to c is lower
        ok = decide16m<FIX>(P, vm, lam, mode, M);
    }
    aff = MARK ? marks16<MARK>(P, okacc, Mlast, c0A, c0B, lam, cap) : okacc * 0xffu;
    return okacc;
}

// Gathers a u16 work item: ra, rb, rc point at the 8-pixel, 16-byte aligned
// block in rows y - 1, y, y + 1; the pixel just left (px == 0) or just right
// (px == 1) of each block must be readable.  wb receives row y's block.
__device__ __forceinline__ void gather_u16(const uint16_t *ra, const uint16_t *rb, const uint16_t *rc, int px, Px16 &P,
                                           uint4 &wb)
{
    // per row: even pixels (0,2) (4,6), odd (1,3) (5,7), and the shifted pairs (-1,1) (3,5) or (2,4) (6,8)
    uint32_t ev[3][2], od[3][2], sh[3][2];
    const uint16_t *rows[3] = {ra, rb, rc};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const uint4 w = *reinterpret_cast<const uint4 *>(rows[r]);
        if (r == 1) wb = w;
        ev[r][0] = __byte_perm(w.x, w.y, 0x5410);
        ev[r][1] = __byte_perm(w.z, w.w, 0x5410);
        od[r][0] = __byte_perm(w.x, w.y, 0x7632);
        od[r][1] = __byte_perm(w.z, w.w, 0x7632);
        if (px == 0) {
            const uint32_t L = *reinterpret_cast<const uint32_t *>(rows[r] - 2);  // pixels -2, -1
            sh[r][0] = __byte_perm(L, w.x, 0x7632);                             // (-1, 1)
            sh[r][1] = __byte_perm(w.y, w.z, 0x7632);                           // (3, 5)
        } else {
            const uint32_t R = *reinterpret_cast<const uint32_t *>(rows[r] + 8);  // pixels 8, 9
            sh[r][0] = __byte_perm(w.y, w.z, 0x5410);                           // (2, 4)
            sh[r][1] = __byte_perm(w.w, R, 0x5410);                             // (6, 8)
        }
    }
    // px == 0: points at the even pixels, E = odd, W = shifted left; px == 1: points at the odd
    // pixels, E = shifted right, W = even.  Ring order E, NE, N, NW, W, SW, S, SE.
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t *nb = h ? P.nbB : P.nbA;
        const uint32_t ctr0 = px ? od[0][h] : ev[0][h], ctr1 = px ? od[1][h] : ev[1][h], ctr2 = px ? od[2][h] : ev[2][h];
        const uint32_t e0 = px ? sh[0][h] : od[0][h], e1 = px ? sh[1][h] : od[1][h], e2 = px ? sh[2][h] : od[2][h];
        const uint32_t w0 = px ? ev[0][h] : sh[0][h], w1 = px ? ev[1][h] : sh[1][h], w2 = px ? ev[2][h] : sh[2][h];
        nb[0] = e1;
        nb[1] = e0;
        nb[2] = ctr0;
        nb[3] = w0;
        nb[4] = w1;
        nb[5] = w2;
        nb[6] = ctr2;
        nb[7] = e2;
        (h ? P.cB : P.cA) = ctr1;
    }
}

// Writes the four points' values back into row y's block.
__device__ __forceinline__ void store_u16(uint16_t *rb, int px, const Px16 &P, uint4 w)
{
    if (px == 0) {
        w.x = __byte_perm(P.cA, w.x, 0x7610);
        w.y = __byte_perm(P.cA, w.y, 0x7632);
        w.z = __byte_perm(P.cB, w.z, 0x7610);
        w.w = __byte_perm(P.cB, w.w, 0x7632);
    } else {
        w.x = __byte_perm(w.x, P.cA, 0x5410);
        w.y = __byte_perm(w.y, P.cA, 0x7610);
        w.z = __byte_perm(w.z, P.cB, 0x5410);
        w.w = __byte_perm(w.w, P.cB, 0x7610);
    }
    *reinterpret_cast<uint4 *>(rb) = w;
}

// One u16 work item under (8,4), tested only: 0x01 in the bytes of the points that would be lowered now.
template <int FIX = -1>
__device__ __forceinline__ uint32_t test_u16(const uint16_t *ra, const uint16_t *rb, const uint16_t *rc, int px,
                                             uint32_t vm, uint32_t lam, int mode)
{
    Px16 P;
    uint4 w;
    gather_u16(ra, rb, rc, px, P, w);
    return decide16m<FIX>(P, vm, lam, mode, lower_mask16(P, P.cA, P.cB));
}

// One u16 work item under (8,4), lowered (ok: a first test's result, or ~0u);
// the block is written back if a point moved.  aff: the neighbours to test again.
template <int FIX = -1, int MARK = 0>
__device__ __forceinline__ uint32_t item_u16(const uint16_t *ra, uint16_t *rb, const uint16_t *rc, int px, uint32_t vm,
                                             uint32_t in, uint32_t ok, uint32_t lam, int mode,
                                             int &nin, uint32_t &aff, bool cap = true)
{
    Px16 P;
    uint4 w;
    gather_u16(ra, rb, rc, px, P, w);
    const uint32_t moved = lower16<FIX, MARK>(P, vm, in, ok, lam, mode, nin, aff, cap);
    if (moved) store_u16(rb, px, P, w);
    return moved;
}

}  // namespace thin
