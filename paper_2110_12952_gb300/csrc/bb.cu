// bb.cu -- the bounding-box approach (Sec. 4, "BB"): the life-like rule on
// every cell of the n^dim box, the baseline the compact step is compared
// with.  Cells off the fractal are dead and are written as 0.
//
// Membership of a box cell factorises over levels: the cell is in the
// fractal iff its lowest Lb base-s digits form a member of the level-Lb
// fractal and its digits above Lb form a member of the level-(r-Lb) one.
// Both are precomputed bitmaps (about sqrt of the box each; the local one
// stores each of its rows twice in a row, so that a run of up to S cells
// starting anywhere in a local row reads as one bit field), so a cell's
// membership costs two divisions by s^Lb = S and two bit look-ups.
//
// Two kernels: bit-sliced rows (bb_bits2_kernel, bb_bits3_kernel, below)
// for boxes of side >= 32 in 16-byte aligned buffers (S >= 32 then); other
// boxes take bb_kernel, where each CTA stages a tile of the box plus a
// one-cell halo in shared memory, one byte per cell (bit 0 = alive member,
// bit 1 = member), and applies the rule from there.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "handle.h"
#include "step.h"

namespace fr {

static int64_t ipow64(int64_t b, int e)
{
    int64_t v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

// membership of a cell of the fractal made of levels base .. base +
// levels - 1 (host, digits by hand)
static bool host_member(const fractal *f, int64_t x, int64_t y, int64_t z, int levels, int base)
{
    for (int mu = 0; mu < levels; ++mu) {
        int t = (int)(x % f->s) + f->s * (int)(y % f->s);
        if (f->dim == 3) t += f->s * f->s * (int)(z % f->s);
        x /= f->s; y /= f->s; z /= f->s;
        if ((f->mixed ? f->lev_hinv[base + mu][t] : f->dev.hinv[t]) < 0) return false;
    }
    return true;
}

// doubled: each row of `side` bits is followed by a copy of itself
static int build_bitmap(const fractal *f, int side, int levels, int base, bool doubled, uint32_t **out, int64_t *words)
{
    const int64_t n = ipow64(side, f->dim), rep = doubled ? 2 : 1;
    const int64_t nw = (n * rep + 31) / 32 + 1;   // one spare word: 32-bit windows may start in the last word
    std::vector<uint32_t> bits(nw, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t x = i % side, y = (i / side) % side, z = f->dim == 3 ? i / ((int64_t)side * side) : 0;
        if (!host_member(f, x, y, z, levels, base)) continue;
        for (int64_t c = 0; c < rep; ++c) {
            const int64_t b = (i / side) * side * rep + c * side + x;
            bits[b >> 5] |= 1u << (b & 31);
        }
    }
    FR_CUDA(cudaMalloc(out, nw * sizeof(uint32_t)));
    FR_CUDA(cudaMemcpy(*out, bits.data(), nw * sizeof(uint32_t), cudaMemcpyHostToDevice));
    *words = nw;
    return FR_OK;
}

void free_bb_plan(BBPlan &p)
{
    cudaFree(p.local_bits);
    cudaFree(p.coarse_bits);
    p = BBPlan();
}

int ensure_bb_plan(fractal *f)
{
    if (f->bb.local_bits) return FR_OK;
    BBPlan p;
    p.Lb = (f->r + 1) / 2;
    while (ipow64(f->s, p.Lb) < 32 && p.Lb < f->r) ++p.Lb;   // S >= 32 where the box allows (bit-sliced rows)
    p.S = (int)ipow64(f->s, p.Lb);
    p.C = (int)ipow64(f->s, f->r - p.Lb);
    int rc = build_bitmap(f, p.S, p.Lb, 0, true, &p.local_bits, &p.local_words);
    if (!rc) rc = build_bitmap(f, p.C, f->r - p.Lb, p.Lb, false, &p.coarse_bits, &p.coarse_words);
    if (rc) {
        free_bb_plan(p);
        return rc;
    }
    f->bb = p;
    return FR_OK;
}

struct BBArgs {
    int32_t n;        // box side
    int32_t S, C;     // local / coarse sides
    DivU32 sdiv;      // division by S
    const uint32_t *local_bits, *coarse_bits;
    int32_t ntx, nty, ntz;   // tiles per axis
    int64_t ntiles;
    uint32_t birth, survive;
};

template <int DIM>
struct BBTile;
template <>
struct BBTile<2> { static constexpr int X = 128, Y = 16, Z = 1; };
template <>
struct BBTile<3> { static constexpr int X = 32, Y = 8, Z = 8; };

__device__ __forceinline__ uint32_t bit_at(const uint32_t *__restrict__ bits, int64_t i)
{
    return (__ldg(bits + (i >> 5)) >> (i & 31)) & 1u;
}

template <int DIM>
__global__ void __launch_bounds__(256)
bb_kernel(BBArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    constexpr int TX = BBTile<DIM>::X, TY = BBTile<DIM>::Y, TZ = BBTile<DIM>::Z;
    constexpr int PX = TX + 2, PY = TY + 2, PZ = (DIM == 3) ? TZ + 2 : 1;
    __shared__ uint8_t tile[PX * PY * PZ];
    const int64_t n = a.n;

    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int tx = (int)(t % a.ntx);
        const int64_t rest = t / a.ntx;
        const int ty = (int)(rest % a.nty);
        const int tz = (int)(rest / a.nty);
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        for (int i = threadIdx.x; i < PX * PY * PZ; i += blockDim.x) {
            const int ix = i % PX, iy = (i / PX) % PY, iz = i / (PX * PY);
            const int gx = x0 - 1 + ix, gy = y0 - 1 + iy, gz = (DIM == 3) ? z0 - 1 + iz : 0;
            uint8_t v = 0;
            if (gx >= 0 && gx < a.n && gy >= 0 && gy < a.n && gz >= 0 && gz < a.n) {
                const uint32_t cx = divu(a.sdiv, gx), cy = divu(a.sdiv, gy), cz = divu(a.sdiv, gz);
                const uint32_t lx = gx - cx * a.S, ly = gy - cy * a.S, lz = gz - cz * a.S;
                const int64_t li = lx + 2 * (int64_t)a.S * (ly + (int64_t)a.S * lz);   // rows stored twice
                const int64_t ci = cx + (int64_t)a.C * (cy + (int64_t)a.C * cz);
                if (bit_at(a.local_bits, li) & bit_at(a.coarse_bits, ci)) {
                    const int64_t g = gx + n * (gy + n * (int64_t)gz);
                    v = 2 | (in[g] != 0);
                }
            }
            tile[i] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < TX * TY * TZ; i += blockDim.x) {
            const int ix = i % TX, iy = (i / TX) % TY, iz = i / (TX * TY);
            const int gx = x0 + ix, gy = y0 + iy, gz = z0 + iz;
            if (gx >= a.n || gy >= a.n || (DIM == 3 && gz >= a.n)) continue;
            const int c = (ix + 1) + PX * ((iy + 1) + PY * (DIM == 3 ? iz + 1 : 0));
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < (DIM == 3 ? 27 : 9); ++q) {
                const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (DIM == 3) ? q / 9 - 1 : 0;
                if (dx == 0 && dy == 0 && dz == 0) continue;
                cnt += tile[c + dx + PX * (dy + PY * dz)] & 1;
            }
            const uint8_t me = tile[c];
            uint8_t v = 0;
            if (me & 2) v = (((me & 1) ? a.survive : a.birth) >> cnt) & 1u;
            out[gx + n * (gy + n * (int64_t)gz)] = v;
        }
        __syncthreads();
    }
}

// 4 bits -> 4 bytes of 0/1 (bit i lands in bit 8i; the other partial
// products fall on distinct non-multiples of 8, so nothing carries)
__device__ __forceinline__ uint32_t nib_bytes(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// 32 bits of a bitmap from bit pos on (bitmaps carry one spare word)
__device__ __forceinline__ uint32_t bits32_at(const uint32_t *__restrict__ bits, uint32_t pos)
{
    return __funnelshift_r(__ldg(bits + (pos >> 5)), __ldg(bits + (pos >> 5) + 1), pos & 31);
}

// the 16 bytes at in + a (a 16-byte aligned), 0 outside [0, total)
__device__ __forceinline__ uint4 load16_bounded(const uint8_t *__restrict__ in, int64_t total, int64_t a)
{
    if (a >= 0 && a + 16 <= total) return __ldg(reinterpret_cast<const uint4 *>(in + a));
    uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const uint32_t b = (a + j >= 0 && a + j < total) ? (uint32_t)__ldg(in + a + j) << (8 * (j & 3)) : 0u;
        if (j < 4) w0 |= b;
        else if (j < 8) w1 |= b;
        else if (j < 12) w2 |= b;
        else w3 |= b;
    }
    return make_uint4(w0, w1, w2, w3);
}

// Bit-sliced rows (bb_bits2_kernel, bb_bits3_kernel; local bitmap side S
// >= 32, box side n >= 32, buffers 16-byte aligned).  A lane owns 32
// consecutive cells x0 .. x0 + 31 of a row (x0 = xs + 32 lane, strips xs
// 992 cells apart) and holds them as one 32-bit word: it loads the 32
// aligned bytes at F + x0 - k (F the row's flat start, k = (F + xs) mod
// 16, the same across the warp), turns each byte into "nonzero" with a
// carry-free multiply, takes the next lane's word and shifts by k, and
// masks with the cells' membership (a 32-bit field of the doubled local
// bitmap row, each part gated by its local tile's coarse bit: at most two
// tiles since S >= 32).  Horizontal 3-sums are two bit planes (full adder of
// the word and its two shifts), the 9 (2D) or 27 (3D) cell totals
// bit-sliced adds of those, and the rule a closed form of the total's bits
// for B3/S23 (2D) and B5/S45 (3D), else a sum over the totals t it maps to
// "alive" of [total == t].  Results go out as aligned 16-byte
// chunks: lane l (0 .. 30) writes the 32 bytes from F + x0 - k + 16 (its
// cells 16 - k .. 31 and the next lane's first ones), which never needs
// lane 0's cell x0 - 1 (unknown unless xs = 0) nor lane 31's last cells
// (their right neighbours lie beyond the warp); strip 0 writes the row's
// head before its first aligned chunk and the chunk holding the row's end
// goes byte by byte, both spread over the lanes.
// 2D: a warp walks kBitsRows2 rows of one strip, four rows at a time.  3D:
// a warp takes kBitsY3 rows of one strip and walks the planes of a chunk of
// `zc` planes, keeping the rows' vertical sums (y - 1 .. y + 1) of the two
// previous planes, so every row is loaded (kBitsY3 + 2) / kBitsY3 times.

constexpr int kBitsStrip = 992;
constexpr int kBitsRows2 = 64;   // a multiple of 4
constexpr int kBitsY3 = 4;

struct BBBitsArgs {
    int32_t n;
    int64_t total;                 // n^dim bytes
    int32_t S, C;
    DivU32 sdiv;
    const uint32_t *local_bits, *coarse_bits;
    int32_t strips, yblocks, zc;   // zc: planes per warp (3D)
    int64_t warps;
    uint32_t amask, dmask;         // bit t: a live / dead cell with total t (self included) lives next
};

struct BitsLane {
    int32_t xs, x0, cx0;
    uint32_t xl0, mask1;           // mask1: the cells in the first local tile (S - xl0 of them)
};

__device__ __forceinline__ BitsLane bits_lane(const BBBitsArgs &a, int32_t sx, int lane)
{
    BitsLane l;
    l.xs = sx * kBitsStrip;
    l.x0 = l.xs + 32 * lane;
    const uint32_t cx = divu(a.sdiv, (uint32_t)l.x0);
    l.cx0 = (int32_t)cx;
    l.xl0 = (uint32_t)l.x0 - cx * (uint32_t)a.S;
    const uint32_t first = (uint32_t)a.S - l.xl0;
    l.mask1 = first >= 32 ? ~0u : (1u << first) - 1u;
    return l;
}

// Where a plane sits: flat offset, its local row (zl S) and coarse row (cz C).
struct BitsPlane {
    int64_t off;
    uint32_t lrow, crow;
    bool live;
};

__device__ __forceinline__ BitsPlane bits_plane(const BBBitsArgs &a, int32_t z)
{
    BitsPlane p;
    p.live = z >= 0 && z < a.n;
    const uint32_t zc = p.live ? (uint32_t)z : 0u, cz = divu(a.sdiv, zc);
    p.off = (int64_t)zc * a.n * a.n;
    p.lrow = (zc - cz * (uint32_t)a.S) * (uint32_t)a.S;
    p.crow = cz * (uint32_t)a.C;
    return p;
}

__device__ __forceinline__ uint32_t coarse_at(const BBBitsArgs &a, uint32_t crow, int32_t cx)
{
    const bool in = cx < a.C;
    const uint32_t c = crow + (uint32_t)(in ? cx : 0);
    return in ? (__ldg(a.coarse_bits + (c >> 5)) >> (c & 31)) & 1u : 0u;
}

// membership of the lane's 32 cells in a row whose (doubled) local bitmap row
// starts at bit `rowbit`, given the coarse bits of the lane's two local tiles
// (bit 0: tile cx0, the cells of mask1; bit 1: tile cx0 + 1)
__device__ __forceinline__ uint32_t member32(const BBBitsArgs &a, const BitsLane &l, uint32_t rowbit, uint32_t cbits)
{
    return bits32_at(a.local_bits, rowbit + l.xl0) & (((cbits & 1u) ? l.mask1 : 0u) | ((cbits & 2u) ? ~l.mask1 : 0u));
}

// the coarse bits of the lane's two local tiles in the coarse row starting at bit `crow`
__device__ __forceinline__ uint32_t coarse2(const BBBitsArgs &a, const BitsLane &l, uint32_t crow)
{
    return coarse_at(a, crow, l.cx0) | (coarse_at(a, crow, l.cx0 + 1) << 1);
}

// bit 7 of each byte: the byte is nonzero
__device__ __forceinline__ uint32_t nz_hi(uint32_t w)
{
    return (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
}

// 32 bytes -> 32 bits (bit i: byte i nonzero).  For two words lo, hi the
// flags sit at bits 3 + 8i (lo, shifted) and 7 + 8i (hi); times 0x204081
// (shifts 0, 7, 14, 21) they land at 24 + i and 28 + i with no two partial
// products on one bit, so no carries: the top byte holds the 8 flags.
__device__ __forceinline__ uint32_t bits32_of(const uint4 &c0, const uint4 &c1)
{
    const uint32_t g0 = ((nz_hi(c0.x) >> 4) | nz_hi(c0.y)) * 0x00204081u;
    const uint32_t g1 = ((nz_hi(c0.z) >> 4) | nz_hi(c0.w)) * 0x00204081u;
    const uint32_t g2 = ((nz_hi(c1.x) >> 4) | nz_hi(c1.y)) * 0x00204081u;
    const uint32_t g3 = ((nz_hi(c1.z) >> 4) | nz_hi(c1.w)) * 0x00204081u;
    return __byte_perm(__byte_perm(g0, g1, 0x7773u), __byte_perm(g2, g3, 0x7773u), 0x5410u);
}

struct H2 {
    uint32_t lo, hi;   // horizontal 3-sums, bit-sliced
};

__device__ __forceinline__ H2 hsum3(uint32_t c, int lane)
{
    uint32_t cp = __shfl_up_sync(0xffffffffu, c, 1);
    const uint32_t cn = __shfl_down_sync(0xffffffffu, c, 1);
    if (lane == 0) cp = 0u;   // cell x0 - 1: outside the box in strip 0, never used otherwise
    const uint32_t lf = __funnelshift_l(cp, c, 1), rt = __funnelshift_r(c, cn, 1);
    return {lf ^ c ^ rt, (lf & c) | (lf & rt) | (c & rt)};
}

// a + b + c of 2-bit values (<= 9): 4 bits
__device__ __forceinline__ void add3_2(const H2 &a, const H2 &b, const H2 &c, uint32_t s[4])
{
    const uint32_t k0 = (a.lo & b.lo) | (a.lo & c.lo) | (b.lo & c.lo);
    const uint32_t u = a.hi ^ b.hi ^ c.hi, v = (a.hi & b.hi) | (a.hi & c.hi) | (b.hi & c.hi);
    s[0] = a.lo ^ b.lo ^ c.lo;
    s[1] = u ^ k0;
    const uint32_t k1 = u & k0;
    s[2] = v ^ k1;
    s[3] = v & k1;
}

__device__ __forceinline__ uint32_t b_maj(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }

// a + b + c of 4-bit values (<= 9 each): 5 bits
__device__ __forceinline__ void add3_4(const uint32_t a[4], const uint32_t b[4], const uint32_t c[4], uint32_t t[5])
{
    t[0] = a[0] ^ b[0] ^ c[0];
    const uint32_t k = b_maj(a[0], b[0], c[0]);                            // weight 2
    const uint32_t u = a[1] ^ b[1] ^ c[1], v = b_maj(a[1], b[1], c[1]);   // v: weight 4
    t[1] = u ^ k;
    const uint32_t w = u & k;                                              // weight 4
    const uint32_t p = a[2] ^ b[2] ^ c[2], q = b_maj(a[2], b[2], c[2]);   // q: weight 8
    t[2] = p ^ v ^ w;
    const uint32_t r = b_maj(p, v, w);                                     // weight 8
    const uint32_t p3 = a[3] ^ b[3] ^ c[3], q3 = b_maj(a[3], b[3], c[3]); // q3: weight 16
    t[3] = p3 ^ q ^ r;
    t[4] = q3 | b_maj(p3, q, r);   // totals stay below 32: never two carries of weight 16
}

// the next state: alive where [total == t] for a t the rule maps to alive
template <int NB>
__device__ __forceinline__ uint32_t rule_bits(const uint32_t t[NB], uint32_t alive, uint32_t amask, uint32_t dmask)
{
    uint32_t r = 0u;
    for (uint32_t u = amask | dmask; u != 0u; u &= u - 1u) {
        const int v = __ffs((int)u) - 1;
        uint32_t eq = ~0u;
#pragma unroll
        for (int i = 0; i < NB; ++i) eq &= ((v >> i) & 1) ? t[i] : ~t[i];
        const uint32_t sa = 0u - ((amask >> v) & 1u), sd = 0u - ((dmask >> v) & 1u);
        r |= eq & ((alive & sa) | (~alive & sd));
    }
    return r;
}

// Rules with a closed form over the total bits: Life B3/S23 in 2D (alive
// next at total 3, or 4 for a live cell) and B5/S45 in 3D (total 5, or 6
// for a live cell); any other rule goes through rule_bits.
constexpr int kRuleAny = 0, kRuleB3S23 = 1, kRuleB5S45 = 2;

template <int NB, int RK>
__device__ __forceinline__ uint32_t rule_of(const uint32_t t[NB], uint32_t alive, uint32_t amask, uint32_t dmask)
{
    if constexpr (RK == kRuleB3S23)
        return ~t[3] & ((~t[2] & t[1] & t[0]) | (alive & t[2] & ~t[1] & ~t[0]));
    else if constexpr (RK == kRuleB5S45)
        return ~t[4] & ~t[3] & t[2] & ((t[0] & ~t[1]) | (alive & t[1] & ~t[0]));
    else
        return rule_bits<NB>(t, alive, amask, dmask);
}

// rows y .. y + NR - 1 of plane p: the lane's cells (masked) and their
// membership; rows outside the box are empty.  FAST: every row is inside
// the box and every window load inside the buffer.
// CACHED: the coarse bits of row j are bits 2j, 2j + 1 of `cb`.
template <int NR, bool FAST, bool CACHED>
__device__ __forceinline__ void bits_rows(const BBBitsArgs &a, const uint8_t *__restrict__ in, const BitsLane &l,
                                          const BitsPlane &p, int32_t y, uint32_t cb, uint32_t c[NR], uint32_t m[NR])
{
    uint4 d0[NR], d1[NR];
    uint32_t k[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int32_t yj = y + j;
        const bool live = FAST || (p.live && yj >= 0 && yj < a.n);
        const int64_t F = p.off + (int64_t)(live ? yj : 0) * a.n;
        k[j] = (uint32_t)((F + l.xs) & 15);
        const int64_t w = F + l.x0 - k[j];
        if (FAST) {
            d0[j] = __ldg(reinterpret_cast<const uint4 *>(in + w));
            d1[j] = __ldg(reinterpret_cast<const uint4 *>(in + w + 16));
        } else if (live) {
            d0[j] = load16_bounded(in, a.total, w);
            d1[j] = load16_bounded(in, a.total, w + 16);
        } else {
            d0[j] = make_uint4(0u, 0u, 0u, 0u);
            d1[j] = d0[j];
        }
        if (live) {
            const uint32_t cy = divu(a.sdiv, (uint32_t)yj);
            const uint32_t yl = (uint32_t)yj - cy * (uint32_t)a.S;
            m[j] = member32(a, l, (p.lrow + yl) * (uint32_t)(2 * a.S),
                            CACHED ? (cb >> (2 * j)) & 3u : coarse2(a, l, (p.crow + cy) * (uint32_t)a.C));
        } else {
            m[j] = 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const uint32_t b = bits32_of(d0[j], d1[j]);
        c[j] = __funnelshift_r(b, __shfl_down_sync(0xffffffffu, b, 1), k[j]) & m[j];
    }
}

// does the window of every lane of rows y .. y + nr - 1 of plane p lie in the box?
__device__ __forceinline__ bool bits_fast(const BBBitsArgs &a, const BitsPlane &p, const BitsLane &l, int32_t y, int nr)
{
    return p.live && y >= 0 && y + nr <= a.n &&
           p.off + (int64_t)(y + nr - 1) * a.n + l.xs + 1024 <= a.total;
}

template <int NR, bool CACHED>
__device__ __forceinline__ void bits_rows_any(const BBBitsArgs &a, const uint8_t *__restrict__ in, const BitsLane &l,
                                              const BitsPlane &p, int32_t y, uint32_t cb, uint32_t c[NR], uint32_t m[NR])
{
    if (bits_fast(a, p, l, y, NR))   // the same in the whole warp
        bits_rows<NR, true, CACHED>(a, in, l, p, y, cb, c, m);
    else
        bits_rows<NR, false, CACHED>(a, in, l, p, y, cb, c, m);
}

// results R of the lane's cells of the row starting at F (see above)
__device__ __forceinline__ void bits_store(uint8_t *__restrict__ out, int64_t F, int32_t n, const BitsLane &l, int lane,
                                           uint32_t R)
{
    const uint32_t k = (uint32_t)((F + l.xs) & 15);
    const int64_t A0 = F + l.xs - k, E = F + n;
    const uint32_t O = __funnelshift_r(R, __shfl_down_sync(0xffffffffu, R, 1), 16u - k);   // bytes A0 + 32 lane + 16 ..
    const int64_t c = A0 + 32 * lane + 16;
    if (lane < 31 && c + 16 <= E)
        *reinterpret_cast<uint4 *>(out + c) =
            make_uint4(nib_bytes(O & 0xfu), nib_bytes((O >> 4) & 0xfu), nib_bytes((O >> 8) & 0xfu), nib_bytes((O >> 12) & 0xfu));
    if (lane < 31 && c + 32 <= E)
        *reinterpret_cast<uint4 *>(out + c + 16) =
            make_uint4(nib_bytes((O >> 16) & 0xfu), nib_bytes((O >> 20) & 0xfu), nib_bytes((O >> 24) & 0xfu), nib_bytes(O >> 28));
    if (l.xs == 0) {   // the row's head: bytes F .. A0 + 15, lane 0's cells 0 .. 15 - k
        const uint32_t h = __shfl_sync(0xffffffffu, R, 0);
        if (lane < 16 - (int)k) out[F + lane] = (uint8_t)((h >> lane) & 1u);
    }
    const int32_t rem = (int32_t)(E & 15);
    if (rem != 0) {   // the chunk holding the row's end, if this strip has it
        const int64_t q = (E - A0 - 16) >> 4;
        if (q >= 0 && q < 62) {
            const uint32_t w = __shfl_sync(0xffffffffu, O, (int)(q >> 1)) >> (16 * (int)(q & 1));
            if (lane < rem) out[A0 + 16 + 16 * q + lane] = (uint8_t)((w >> lane) & 1u);
        }
    }
}

template <int RK>
__global__ void __launch_bounds__(128)
bb_bits2_kernel(BBBitsArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= a.warps) return;   // whole warps leave together
    const BitsLane l = bits_lane(a, (int32_t)(wid % a.strips), lane);
    const int32_t y0 = (int32_t)(wid / a.strips) * kBitsRows2, y1 = min(y0 + kBitsRows2, a.n);
    const BitsPlane p = bits_plane(a, 0);
    // Hm, H0: sums of rows y - 1, y; c0, m0: row y
    uint32_t c[4], m[4];
    bits_rows<2, false, false>(a, in, l, p, y0 - 1, 0u, c, m);
    H2 Hm = hsum3(c[0], lane), H0 = hsum3(c[1], lane);
    uint32_t c0 = c[1], m0 = m[1];
    for (int32_t y = y0; y < y1; y += 4) {
        bits_rows_any<4, false>(a, in, l, p, y + 1, 0u, c, m);
        const H2 h[6] = {Hm, H0, hsum3(c[0], lane), hsum3(c[1], lane), hsum3(c[2], lane), hsum3(c[3], lane)};
        const uint32_t cc[4] = {c0, c[0], c[1], c[2]}, mm[4] = {m0, m[0], m[1], m[2]};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (y + i >= y1) break;   // the same in the whole warp
            uint32_t t[4];
            add3_2(h[i], h[i + 1], h[i + 2], t);
            const uint32_t R = rule_of<4, RK>(t, cc[i], a.amask, a.dmask) & mm[i];
            bits_store(out, (int64_t)(y + i) * a.n, a.n, l, lane, R);
        }
        Hm = h[4];
        H0 = h[5];
        c0 = c[3];
        m0 = m[3];
    }
}

// vertical sums of rows y0 .. y0 + kBitsY3 - 1 of plane z, with the rows' cells
// and membership (cb: the coarse bits of rows y0 - 1 .. y0 + kBitsY3)
__device__ __forceinline__ void bits3_plane(const BBBitsArgs &a, const uint8_t *__restrict__ in, const BitsLane &l,
                                            int lane, int32_t z, int32_t y0, uint32_t cb, uint32_t V[kBitsY3][4],
                                            uint32_t cen[kBitsY3], uint32_t mem[kBitsY3])
{
    constexpr int NR = kBitsY3 + 2;
    uint32_t c[NR], m[NR];
    const BitsPlane p = bits_plane(a, z);
    bits_rows_any<NR, true>(a, in, l, p, y0 - 1, cb, c, m);
    H2 h[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) h[j] = hsum3(c[j], lane);
#pragma unroll
    for (int i = 0; i < kBitsY3; ++i) {
        add3_2(h[i], h[i + 1], h[i + 2], V[i]);
        cen[i] = c[i + 1];
        mem[i] = m[i + 1];
    }
}

template <int RK>
__global__ void __launch_bounds__(128, 4)
bb_bits3_kernel(BBBitsArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= a.warps) return;   // whole warps leave together
    const BitsLane l = bits_lane(a, (int32_t)(wid % a.strips), lane);
    const int64_t rest = wid / a.strips;
    const int32_t y0 = (int32_t)(rest % a.yblocks) * kBitsY3;
    const int32_t zb = (int32_t)(rest / a.yblocks) * a.zc, ze = min(zb + a.zc, a.n);
    // planes z - 1 (Vm) and z (V0, c0, m0) around the plane z being written
    uint32_t Vm[kBitsY3][4] = {}, V0[kBitsY3][4] = {}, c0[kBitsY3] = {}, m0[kBitsY3] = {};
    uint32_t cb = 0u;      // coarse bits of rows y0 - 1 .. y0 + kBitsY3 in coarse plane cb_cz
    int32_t cb_cz = -1;
    for (int32_t q = zb - 1; q <= ze; ++q) {
        const int32_t cz = q >= 0 && q < a.n ? (int32_t)divu(a.sdiv, (uint32_t)q) : -1;
        if (cz >= 0 && cz != cb_cz) {   // the same in the whole warp
            cb = 0u;
#pragma unroll
            for (int j = 0; j < kBitsY3 + 2; ++j) {
                const int32_t y = y0 - 1 + j;
                if (y >= 0 && y < a.n)
                    cb |= coarse2(a, l, ((uint32_t)cz * (uint32_t)a.C + divu(a.sdiv, (uint32_t)y)) * (uint32_t)a.C) << (2 * j);
            }
            cb_cz = cz;
        }
        uint32_t Vp[kBitsY3][4], cp[kBitsY3], mp[kBitsY3];
        bits3_plane(a, in, l, lane, q, y0, cb, Vp, cp, mp);
        if (q > zb) {   // write plane q - 1
            const int64_t base = (int64_t)(q - 1) * a.n * a.n;
#pragma unroll
            for (int i = 0; i < kBitsY3; ++i) {
                if (y0 + i >= a.n) break;   // the same in the whole warp
                uint32_t t[5];
                add3_4(Vm[i], V0[i], Vp[i], t);
                const uint32_t R = rule_of<5, RK>(t, c0[i], a.amask, a.dmask) & m0[i];
                bits_store(out, base + (int64_t)(y0 + i) * a.n, a.n, l, lane, R);
            }
        }
#pragma unroll
        for (int i = 0; i < kBitsY3; ++i) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                Vm[i][b] = V0[i][b];
                V0[i][b] = Vp[i][b];
            }
            c0[i] = cp[i];
            m0[i] = mp[i];
        }
    }
}

int launch_bb_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                   uint32_t survive, cudaStream_t st)
{
    if (f->bb.S >= 32 && f->side >= 32 && ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        const BBPlan &p = f->bb;
        BBBitsArgs a;
        a.n = (int32_t)f->side;
        a.total = (int64_t)f->side * f->side * (f->dim == 3 ? f->side : 1);
        a.S = p.S;
        a.C = p.C;
        a.sdiv = make_div((uint32_t)p.S);
        a.local_bits = p.local_bits;
        a.coarse_bits = p.coarse_bits;
        // strip sx writes cells up to 992 sx + 1008 - k (k < 16), strip 0 from cell 0 on
        a.strips = a.n <= 993 ? 1 : (a.n - 993 + 991) / 992 + 1;
        if (f->dim == 3) {
            a.amask = (survive << 1) & 0x0ffffffeu;
            a.dmask = birth & 0x07ffffffu;
            a.yblocks = (a.n + kBitsY3 - 1) / kBitsY3;
            // chunks of planes so that the warps fill the GPU once (as far as n allows)
            int blocks = 0;
            FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, bb_bits3_kernel<kRuleAny>, 128, 0));
            const int64_t cols = (int64_t)a.strips * a.yblocks;
            const int64_t chunks = std::max<int64_t>(1, (int64_t)std::max(blocks, 1) * 4 * f->num_sms / cols);
            a.zc = (int32_t)((a.n + chunks - 1) / chunks);
            a.warps = cols * ((a.n + a.zc - 1) / a.zc);
        } else {
            a.amask = (survive << 1) & 0x3feu;
            a.dmask = birth & 0x1ffu;
            a.yblocks = (a.n + kBitsRows2 - 1) / kBitsRows2;
            a.zc = 1;
            a.warps = (int64_t)a.strips * a.yblocks;
        }
        const int64_t grid = (a.warps + 3) / 4;
        if (f->dim == 3 && a.amask == 0x60u && a.dmask == 0x20u)
            bb_bits3_kernel<kRuleB5S45><<<(unsigned)grid, 128, 0, st>>>(a, in, out);
        else if (f->dim == 3)
            bb_bits3_kernel<kRuleAny><<<(unsigned)grid, 128, 0, st>>>(a, in, out);
        else if (a.amask == 0x18u && a.dmask == 0x8u)
            bb_bits2_kernel<kRuleB3S23><<<(unsigned)grid, 128, 0, st>>>(a, in, out);
        else
            bb_bits2_kernel<kRuleAny><<<(unsigned)grid, 128, 0, st>>>(a, in, out);
        FR_CUDA(cudaGetLastError());
        return FR_OK;
    }
    const BBPlan &p = f->bb;
    BBArgs a;
    a.n = (int32_t)f->side;
    a.S = p.S;
    a.C = p.C;
    a.sdiv = make_div((uint32_t)std::max(p.S, 2));
    a.local_bits = p.local_bits;
    a.coarse_bits = p.coarse_bits;
    a.birth = birth;
    a.survive = survive;
    int tx, ty, tz;
    if (f->dim == 2) {
        tx = BBTile<2>::X; ty = BBTile<2>::Y; tz = 1;
    } else {
        tx = BBTile<3>::X; ty = BBTile<3>::Y; tz = BBTile<3>::Z;
    }
    a.ntx = (int32_t)((f->side + tx - 1) / tx);
    a.nty = (int32_t)((f->side + ty - 1) / ty);
    a.ntz = f->dim == 3 ? (int32_t)((f->side + tz - 1) / tz) : 1;
    a.ntiles = (int64_t)a.ntx * a.nty * a.ntz;
    int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)f->num_sms * 8);
    if (f->dim == 2)
        bb_kernel<2><<<(int)grid, 256, 0, st>>>(a, in, out);
    else
        bb_kernel<3><<<(int)grid, 256, 0, st>>>(a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

}  // namespace fr
