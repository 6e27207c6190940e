// bit3.cuh -- the "bit3" policy of the compact step for 3D fractals with
// s = 3 and k a multiple of 4 (the Menger sponge, k = 20): one warp per
// level-3 tile and no block barriers.  The tile's 27^3 box with its one-cell
// halo is held bit-sliced, one 32-bit word per box row (y, z): bit x + 1 is
// cell x, bits 0 and 28 are the halo cells.  The 27-cell totals of the
// 26-neighbour rule (Sec. 3 stencil, in three dimensions) are carry-save
// adders on whole rows: the x-sums of a row from two shifts and a full
// adder, the y-sums across the warp's lanes (lane = y) by shuffles, the
// z-sums slid down z in registers.  Included by step.cu after its helpers.
//
// Per tile the warp
//   1. fetches the halo: the level-1 blocks of the existing neighbour tiles
//      that touch the box's one-cell ring, converted as in 2 and cut to the
//      ring;
//   2. turns the tile's cells into box bits.  A level-1 block is k bytes
//      (consecutive in omega) filling a 3x3x3 cube; four cells of a word
//      become a nibble through a carry-free multiply, a table maps each
//      word's nibble to its cube bits, and the cube's 3-bit row pieces are
//      ORed into the box rows (shared-memory atomics: up to nine blocks share
//      a row);
//   3. replaces the inner rows by the next generation, walking down z;
//   4. reads each block's row pieces back, a table maps them to the block's
//      k result bits in the tile's bit string, and a multiply spreads each
//      nibble of that string into four bytes.
// Each lane reads its blocks' words straight from memory, one block ahead
// (the first while the halo is fetched); with a small shared-memory area per
// warp, 32 warps fit on an SM to hide the latency.  The results are gathered
// into a bit string in omega order and leave as whole 16-byte words.
//
// A call of several generations keeps the state bit-packed between them
// (bit3_layout.h: per tile its inner rows and its two x-faces): the first
// generation does 1-3 and writes rows and faces, the last reads the rows in
// 3 from the states and does 4, the ones between do neither conversion.
#pragma once

#include <stdint.h>

#include "bit3_layout.h"

namespace fr {

__device__ __forceinline__ uint32_t b3_xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }
__device__ __forceinline__ uint32_t b3_maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }

// A count per bit position, bit-sliced: value = b0 + 2 b1 + 4 b2 + 8 b3.
struct B3Q {
    uint32_t b0, b1, b2, b3;
};
// The same with five slices (totals <= 27).
struct B3T {
    uint32_t t0, t1, t2, t3, t4;
};

// Sums over x and y of the 3x3 cells around each cell of row (lane, z): the
// row's x-sums (0..3) from its own word, added to those of rows y - 1 and
// y + 1 (the neighbouring lanes).  Lanes 0 and 28 (halo rows) get values
// that are never used.
__device__ __forceinline__ B3Q b3_sxy(uint32_t w)
{
    const uint32_t l = w << 1, r = w >> 1;
    const uint32_t s0 = b3_xor3(l, w, r), s1 = b3_maj3(l, w, r);
    const uint32_t u0 = __shfl_up_sync(0xffffffffu, s0, 1), u1 = __shfl_up_sync(0xffffffffu, s1, 1);
    const uint32_t d0 = __shfl_down_sync(0xffffffffu, s0, 1), d1 = __shfl_down_sync(0xffffffffu, s1, 1);
    B3Q q;
    q.b0 = b3_xor3(u0, s0, d0);
    const uint32_t k1 = b3_maj3(u0, s0, d0);                              // weight 2
    const uint32_t v1 = b3_xor3(u1, s1, d1), v2 = b3_maj3(u1, s1, d1);    // weights 2, 4
    q.b1 = k1 ^ v1;
    const uint32_t k2 = k1 & v1;                                          // weight 4
    q.b2 = v2 ^ k2;
    q.b3 = v2 & k2;
    return q;
}

// a + b + c for three counts <= 9 (carry-save, ripple over the weights)
__device__ __forceinline__ B3T b3_add3(const B3Q &a, const B3Q &b, const B3Q &c)
{
    B3T t;
    t.t0 = b3_xor3(a.b0, b.b0, c.b0);
    const uint32_t c1 = b3_maj3(a.b0, b.b0, c.b0);                              // 2
    const uint32_t x1 = b3_xor3(a.b1, b.b1, c.b1), y2 = b3_maj3(a.b1, b.b1, c.b1);  // 2, 4
    t.t1 = x1 ^ c1;
    const uint32_t z2 = x1 & c1;                                                // 4
    const uint32_t p2 = b3_xor3(a.b2, b.b2, c.b2), q3 = b3_maj3(a.b2, b.b2, c.b2);  // 4, 8
    t.t2 = b3_xor3(p2, y2, z2);
    const uint32_t r3 = b3_maj3(p2, y2, z2);                                    // 8
    const uint32_t m3 = b3_xor3(a.b3, b.b3, c.b3), n4 = b3_maj3(a.b3, b.b3, c.b3);  // 8, 16
    t.t3 = b3_xor3(m3, q3, r3);
    t.t4 = n4 | b3_maj3(m3, q3, r3);   // one weight-16 carry at most: totals are <= 27
    return t;
}

template <int V>
__device__ __forceinline__ uint32_t b3_eq(const B3T &t)
{
    const uint32_t a = (V & 1) ? t.t0 : ~t.t0, b = (V & 2) ? t.t1 : ~t.t1, c = (V & 4) ? t.t2 : ~t.t2;
    const uint32_t d = (V & 8) ? t.t3 : ~t.t3, e = (V & 16) ? t.t4 : ~t.t4;
    return a & b & c & d & e;
}

// positions whose total equals v (v is the same in every lane)
__device__ __forceinline__ uint32_t b3_eq_rt(int v, const B3T &t)
{
    switch (v) {
#define FR_B3_EQ(V) case V: return b3_eq<V>(t);
        FR_B3_EQ(0) FR_B3_EQ(1) FR_B3_EQ(2) FR_B3_EQ(3) FR_B3_EQ(4) FR_B3_EQ(5) FR_B3_EQ(6)
        FR_B3_EQ(7) FR_B3_EQ(8) FR_B3_EQ(9) FR_B3_EQ(10) FR_B3_EQ(11) FR_B3_EQ(12) FR_B3_EQ(13)
        FR_B3_EQ(14) FR_B3_EQ(15) FR_B3_EQ(16) FR_B3_EQ(17) FR_B3_EQ(18) FR_B3_EQ(19) FR_B3_EQ(20)
        FR_B3_EQ(21) FR_B3_EQ(22) FR_B3_EQ(23) FR_B3_EQ(24) FR_B3_EQ(25) FR_B3_EQ(26) FR_B3_EQ(27)
#undef FR_B3_EQ
        default: return 0u;
    }
}

// The life-like rule on totals that count the cell itself: a dead cell is
// born at a total in `bonly` or `both`, a live cell survives at one in
// `sonly` or `both` (masks of totals 0..27).
__device__ __forceinline__ uint32_t b3_rule(const B3T &t, uint32_t alive, uint32_t both, uint32_t sonly,
                                            uint32_t bonly)
{
    uint32_t e = 0u, es = 0u, eb = 0u;
    for (uint32_t m = both; m; m &= m - 1) e |= b3_eq_rt(__ffs(m) - 1, t);
    for (uint32_t m = sonly; m; m &= m - 1) es |= b3_eq_rt(__ffs(m) - 1, t);
    for (uint32_t m = bonly; m; m &= m - 1) eb |= b3_eq_rt(__ffs(m) - 1, t);
    return e | (alive & es) | (~alive & eb);
}

// The words of the level-1 block at src (k bytes, k = 4 kw): aligned
// 4-byte loads, or bytes where the buffer is not 4-byte aligned.
template <int KW>
__device__ __forceinline__ void b3_load_block(uint32_t (&w)[6], const uint8_t *src, int kw, bool al4,
                                              uint32_t wmask = 0x3fu)
{
#pragma unroll
    for (int q = 0; q < (KW ? KW : 6); ++q) {
        w[q] = 0u;
        if ((KW || q < kw) && ((wmask >> q) & 1u)) {
            if (al4)
                w[q] = __ldg(reinterpret_cast<const uint32_t *>(src) + q);
            else
                w[q] = __ldg(src + 4 * q) | (uint32_t)__ldg(src + 4 * q + 1) << 8 |
                       (uint32_t)__ldg(src + 4 * q + 2) << 16 | (uint32_t)__ldg(src + 4 * q + 3) << 24;
        }
    }
}

// The 27-bit cube of a block (bit x + 3y + 9z for its cell at (x, y, z))
// from its words (those in wmask): bit 7 of each nonzero byte, bits 7, 15,
// 23, 31 gathered into a nibble by a carry-free multiply, a table per word
// and nibble.
template <int KW>
__device__ __forceinline__ uint32_t b3_cube(const uint32_t (&w)[6], const uint32_t *CT, int kw, uint32_t wmask = 0x3fu)
{
    uint32_t cube = 0u;
#pragma unroll
    for (int q = 0; q < (KW ? KW : 6); ++q) {
        if ((KW || q < kw) && ((wmask >> q) & 1u)) {
            const uint32_t c = (((w[q] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w[q]) & 0x80808080u;
            cube |= CT[q * 16 + ((c * 0x00204081u) >> 28)];
        }
    }
    return cube;
}

// 4 bits -> 4 bytes of 0/1 (bit i lands in bit 8i; the other partial
// products fall on distinct non-multiples of 8, so nothing carries)
__device__ __forceinline__ uint32_t b3_nib_bytes(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// All-zero bit state standing in for absent neighbour tiles.
__device__ __align__(16) uint32_t g_b3_zero_state[kB3StateWords];

// Box row (y, z) (0..28 each) of a tile from bit-packed states: its cells from the
// row of the tile (or of the neighbour across the ring) that holds them,
// its ring bits 0 and 28 from the x-faces of the neighbours in x.  st[q] is
// the state of the tile in direction q = (dx + 1) + 3 (dy + 1) + 9 (dz + 1)
// (13: the tile itself; absent tiles: zeros).
__device__ __forceinline__ uint32_t b3_row_from_state(const uint32_t *const *st, int y, int z)
{
    const int dy = (y == 0) ? -1 : (y == 28 ? 1 : 0), dz = (z == 0) ? -1 : (z == 28 ? 1 : 0);
    const int sy = y - 27 * dy - 1, sz = z - 27 * dz - 1;   // the cell row in the tile that holds it, 0..26
    const int q = 13 + 3 * dy + 9 * dz;                     // direction (0, dy, dz), 1..25
    uint32_t w = __ldg(st[q] + sy + 27 * sz);
    w |= (__ldg(st[q - 1] + kB3StateXH + sz) >> sy) & 1u;            // cell x = -1: face x = 26 of the -x tile
    w |= ((__ldg(st[q + 1] + kB3StateXL + sz) >> sy) & 1u) << 28;    // cell x = 27: face x = 0 of the +x tile
    return w;
}

// B5S45: the rule is B5/S45 (totals 5 for birth, 5 and 6 for survival),
// evaluated with constants; otherwise the rule of the tile's instance.
// KW: words per level-1 block (k / 4), or 0 when read from the arguments.
// IN_BITS / OUT_BITS: the generation reads / writes the bit-packed states
// a.b3.sin / a.b3.sout instead of bytes (single-instance launches).
template <bool MULTI, bool B5S45, int KW, bool IN_BITS = false, bool OUT_BITS = false>
__global__ void __launch_bounds__(32 * kB3Warps, (IN_BITS && OUT_BITS && B5S45) ? 5 : 4)
step_bit3_kernel(StepArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *stab = reinterpret_cast<uint32_t *>(smem);
    for (int i = threadIdx.x; i < a.b3.nshared; i += blockDim.x) stab[i] = __ldg(a.tab + i);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // states -> states needs no box and no result bits, only each warp's 27
    // state pointers (kB3StatePtrBytes): five blocks fit per SM
    constexpr bool kStatesOnly = IN_BITS && OUT_BITS;
    uint8_t *wb = smem + a.b3.off_warp + warp * (kStatesOnly ? kB3StatePtrBytes : a.b3.warp_bytes);
    uint32_t *box = reinterpret_cast<uint32_t *>(wb);
    const uint8_t **nbase = reinterpret_cast<const uint8_t **>(wb + (kStatesOnly ? 0 : kB3OffPtr));
    uint32_t *bits = reinterpret_cast<uint32_t *>(wb + kB3OffBits);
    const uint32_t *CT = stab, *RT = stab + a.b3.off_rt, *BP = stab + a.b3.off_bp, *HS = stab + a.b3.off_hs;
    const uint2 *HE = reinterpret_cast<const uint2 *>(stab + a.b3.off_he);
    const int k = KW ? 4 * KW : a.b3.k, kw = KW ? KW : k / 4, nblk = k * k;
    const int64_t KL = a.KL, stride = (int64_t)gridDim.x * kB3Warps;
    const int nbw = (int)(KL / 32);

    for (int64_t Tg = (int64_t)blockIdx.x * kB3Warps + warp; Tg < a.NT; Tg += stride) {
        const TileRef t = resolve<MULTI>(a, in, out, Tg);
        Rule rule;
        tile_rule<MULTI>(a, Tg, rule);
        const uint32_t mb = rule.birth & 0x7ffffffu, ms = (rule.survive << 1) & 0xffffffeu;
        const uint32_t both = mb & ms, sonly = ms & ~mb, bonly = mb & ~ms;
        uint8_t *tout = t.out + t.T * KL;
        const uint8_t *tin = t.in + t.T * KL;
        const int32_t tn = lane < 26 ? __ldg(t.nbr + t.T * a.nbrw + lane) : -1;
        if constexpr (IN_BITS) {
            // 1-2. the states of the tile and its neighbours, by direction; the
            // rows are read from them as the walk below needs them
            const uint32_t **st = reinterpret_cast<const uint32_t **>(nbase);
            const int32_t tq = __shfl_sync(0xffffffffu, tn, lane < 13 ? lane : lane - 1);   // direction lane -> slot
            if (lane < 27)
                st[lane] = lane == 13 ? a.b3.sin + t.T * kB3StateWords
                                      : (tq >= 0 ? a.b3.sin + (int64_t)tq * kB3StateWords : g_b3_zero_state);
            __syncwarp();
        } else {
            const bool al4 = (((uintptr_t)t.in) & 3) == 0;
            // the lane's first block of the tile, loaded while the halo is fetched
            uint32_t wn[6];
            if (lane < nblk) b3_load_block<KW>(wn, tin + k * lane, kw, al4);
            // neighbour tiles by slot
            const uint32_t present = __ballot_sync(0xffffffffu, tn >= 0);
            if (lane < 26) nbase[lane] = tn >= 0 ? t.in + (int64_t)tn * KL : t.in;

            // 1. the halo: the blocks of the neighbour tiles that touch the box's
            // halo ring, converted like the tile's own blocks, their row pieces
            // cut to the ring (entries grouped by neighbour slot; absent tiles
            // are skipped)
            for (int i = lane; i < kB3BoxWords / 4; i += 32) reinterpret_cast<uint4 *>(box)[i] = make_uint4(0, 0, 0, 0);
            __syncwarp();
            for (uint32_t pm = present & 0x3ffffffu; pm; pm &= pm - 1) {
                const int d = __ffs(pm) - 1;
                const uint32_t hs = HS[d], wm = hs >> 26;   // the words holding the cells this direction needs
                const uint8_t *nt = nbase[d];
                for (int e = (int)(hs & 0x1fffu) + lane; e < (int)((hs >> 13) & 0x1fffu); e += 32) {
                    const uint2 en = HE[e];
                    uint32_t w[6];
                    b3_load_block<KW>(w, nt + k * (int)((en.x >> 5) & 1023u), kw, al4, wm);
                    const uint32_t cube = b3_cube<KW>(w, CT, kw, wm);
                    const uint32_t rmask = (en.x >> 15) & 511u, pmask = (en.x >> 24) & 7u, sh2 = en.x >> 27;
                    const int rb = (int)en.y;
#pragma unroll
                    for (int rr = 0; rr < 9; ++rr)
                        if ((rmask >> rr) & 1u)
                            atomicOr(&box[rb + rr % 3 + kB3Pitch * (rr / 3)], (((cube >> (3 * rr)) & pmask) << sh2) >> 2);
                }
            }
            // 2. the tile's cells, a block per lane (the next one loaded ahead),
            // ORed into their rows
            for (int j = lane; j < nblk; j += 32) {
                uint32_t wc[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) wc[q] = wn[q];
                if (j + 32 < nblk) b3_load_block<KW>(wn, tin + k * (j + 32), kw, al4);
                const uint32_t cube = b3_cube<KW>(wc, CT, kw);
                const uint32_t bp = BP[j];
                const int rb = (int)(bp & 0xffffu), sh = (int)(bp >> 16);
#pragma unroll
                for (int rr = 0; rr < 9; ++rr)
                    if ((a.b3.rowset >> rr) & 1u)   // rows of the cube that hold members
                        atomicOr(&box[rb + rr % 3 + kB3Pitch * (rr / 3)], ((cube >> (3 * rr)) & 7u) << sh);
            }
            __syncwarp();
        }
        // the result bits start at zero (ORed into below)
        if constexpr (!OUT_BITS)
            for (int i = lane; i < nbw; i += 32) bits[i] = 0u;

        // 3. the next generation of the inner rows, in place: step z reads
        // row z and writes row z - 1, whose sums are already in registers
        {
            // box row (lane, z): from the box, or (bit states) from the states;
            // in the planes 1..27 a lane's row and its ring bits come from the
            // same three states, fixed for the tile
            const uint32_t *const *st = reinterpret_cast<const uint32_t *const *>(nbase);
            const int dyl = lane == 0 ? -1 : (lane == 28 ? 1 : 0), syl = lane - 27 * dyl - 1;
            const uint32_t *p0 = nullptr, *pm = nullptr, *pp = nullptr;
            if constexpr (IN_BITS) {
                if (lane < kB3Pitch) {
                    p0 = st[13 + 3 * dyl] + syl;
                    pm = st[12 + 3 * dyl] + kB3StateXH;
                    pp = st[14 + 3 * dyl] + kB3StateXL;
                }
            }
            auto row = [&](int z) -> uint32_t {
                if (lane >= kB3Pitch) return 0u;
                if constexpr (IN_BITS) {
                    if (z == 0 || z == kB3Pitch - 1) return b3_row_from_state(st, lane, z);
                    const int sz = z - 1;
                    return __ldg(p0 + 27 * sz) | ((__ldg(pm + sz) >> syl) & 1u) | (((__ldg(pp + sz) >> syl) & 1u) << 28);
                } else {
                    return box[lane + kB3Pitch * z];
                }
            };
            const uint32_t w0 = row(0), w1 = row(1);
            B3Q qa = b3_sxy(w0), qb = b3_sxy(w1);
            // rows three planes ahead are in flight (reads from the states
            // come from L2)
            uint32_t alive = w1, wa = row(2), wb = row(3), wc = row(4);
#pragma unroll 3
            for (int z = 2; z < kB3Pitch; ++z) {
                const uint32_t w = wa;
                wa = wb;
                wb = wc;
                wc = (z + 3 < kB3Pitch) ? row(z + 3) : 0u;
                const B3Q qc = b3_sxy(w);
                const B3T tt = b3_add3(qa, qb, qc);
                uint32_t nw;
                if constexpr (B5S45)
                    nw = b3_eq<5>(tt) | (alive & b3_eq<6>(tt));
                else
                    nw = b3_rule(tt, alive, both, sonly, bonly);
                const bool inner = lane >= 1 && lane <= 27;
                if constexpr (OUT_BITS) {
                    // the new row and the row's cells x = 0 and x = 26 into the faces
                    uint32_t *so = a.b3.sout + t.T * kB3StateWords;
                    // (positions off the fractal dropped: the next generation reads these rows whole)
                    if (inner) nw &= stab[a.b3.off_mr + (lane - 1) + 27 * (z - 2)];
                    if (inner) so[(lane - 1) + 27 * (z - 2)] = nw;
                    const uint32_t xl = __ballot_sync(0xffffffffu, inner && ((nw >> 1) & 1u)) >> 1;
                    const uint32_t xh = __ballot_sync(0xffffffffu, inner && ((nw >> 27) & 1u)) >> 1;
                    if (lane == 0) {
                        so[kB3StateXL + z - 2] = xl;
                        so[kB3StateXH + z - 2] = xh;
                    }
                } else {
                    if (inner) box[lane + kB3Pitch * (z - 1)] = nw & 0x0ffffffeu;
                }
                qa = qb;
                qb = qc;
                alive = w;
            }
        }
        __syncwarp();

        if constexpr (!OUT_BITS) {
            // 4. the results: each block's k bits (a table per row piece) into
            // the tile's bit string, then 16 cells per lane and step to memory
            for (int j = lane; j < nblk; j += 32) {
                const uint32_t bp = BP[j];
                const int rb = (int)(bp & 0xffffu), sh = (int)(bp >> 16);
                uint32_t m = 0u;
#pragma unroll
                for (int rr = 0; rr < 9; ++rr)
                    if ((a.b3.rowset >> rr) & 1u)
                        m |= RT[rr * 8 + ((box[rb + rr % 3 + kB3Pitch * (rr / 3)] >> sh) & 7u)];
                const int b = k * j, wi = b >> 5, s = b & 31;
                atomicOr(&bits[wi], m << s);
                if (s + k > 32) atomicOr(&bits[wi + 1], m >> (32 - s));
            }
            __syncwarp();
            if ((((uintptr_t)tout) & 15) == 0) {
                for (int h = lane; h < (int)(KL / 16); h += 32) {
                    const uint32_t hw = bits[h >> 1] >> (16 * (h & 1));
                    reinterpret_cast<uint4 *>(tout)[h] =
                        make_uint4(b3_nib_bytes(hw & 0xfu), b3_nib_bytes((hw >> 4) & 0xfu), b3_nib_bytes((hw >> 8) & 0xfu),
                                   b3_nib_bytes((hw >> 12) & 0xfu));
                }
            } else {
                for (int c = lane; c < (int)KL; c += 32) tout[c] = (uint8_t)((bits[c >> 5] >> (c & 31)) & 1u);
            }
            __syncwarp();
        }
    }
}

}  // namespace fr
