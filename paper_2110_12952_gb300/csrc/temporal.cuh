// temporal.cuh -- temporal blocking of the compact step for the carpet and
// the Vicsek fractal (the fractals of rows_layout.h): one pass over the state
// advances every cell by up to 9 generations.  Included at the end of
// step.cu (it uses the rows policy's compile-time unit layout).
//
// A tile (level-L subtree, k^L cells) and the level-2 units of its 8
// neighbouring tiles that touch it (a ring one unit, 9 cells, wide) are
// loaded once, turned into a bitmap box of (3^L + 18)^2 cells with one bit
// per cell (32 cells per word, rows padded by a zero guard word on each
// side), advanced g <= 9 generations there with bit-sliced arithmetic, and
// the tile's cells are written back in omega order.  Generation j computes
// the rows at distance >= j from the box edge only: a cell at distance d is
// exact after min(d, g) generations, and the tile's cells are at distance
// >= 9.  A second bitmap holds the members of the box (the unit pattern of
// every present unit; nothing for holes and for absent neighbouring tiles),
// and every generation's result is masked with it, so non-members stay dead.
//
// Per generation and 32 box cells: 3 word loads (a thread walks down a word
// column keeping three rows in registers), 6 funnel shifts for the west/east
// neighbours, 14 logic operations for the 8-input bit-sliced adder (count
// bits b3..b0), the rule (3 for B3/S23, else 17: a multiplexer tree over the
// count bits with the birth/survival tables as all-ones or all-zero words),
// the mask and a store.  HBM bytes per cell-update: (tile + halo
// units + tile) / (tile cells x generations) instead of 2.
#pragma once

namespace fr {

struct TbArgs {
    int64_t KL, NT;
    int nu;          // units per tile
    int nring;       // halo units per tile
    int W;           // box side in cells
    int RS;          // words per box row: NWB data words and two zero guards
    int NWB;
    int gens;
    uint32_t birth, survive;
    const uint16_t *upos;   // tile unit q -> box unit position (x | y << 8), ring included
    const uint32_t *ring;   // halo unit e: [2e] unit index in the neighbouring tile | slot << 24, [2e+1] box unit position
    const int32_t *nbr;     // per tile: 8 neighbouring tiles, -1 none
    int off_halo, off_pres, off_box0, off_box1, off_mask;
    int *status;
};

// bit x of the result = the byte of column x - 1 .. x + 2 (word w) being 1
__device__ __forceinline__ uint32_t tb_nibble(uint32_t w) { return (w * 0x01020408u) >> 24; }
__device__ __forceinline__ uint32_t tb_expand4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }
__device__ __forceinline__ uint32_t tb_sel(uint32_t c, uint32_t a, uint32_t b) { return (c & a) | (~c & b); }

// membership pattern of row y (0..8) of a unit's 9x9 block: bit x set for a member
template <int P>
constexpr uint32_t tb_pattern(int y)
{
    uint32_t m = 0;
    for (int x = 0; x < 9; ++x)
        if (rp_byte<P>(x, y) >= 0) m |= 1u << x;
    return m;
}

// OR the 9-bit row segment `bits` into box row Y at cell column X
__device__ __forceinline__ void tb_or_bits(uint32_t *box, int RS, int Y, int X, uint32_t bits)
{
    uint32_t *row = box + Y * RS + 1 + (X >> 5);
    const int sh = X & 31;
    atomicOr(row, bits << sh);
    if (sh > 23) atomicOr(row + 1, bits >> (32 - sh));
}

__device__ __forceinline__ uint32_t tb_get_bits(const uint32_t *box, int RS, int Y, int X)
{
    const uint32_t *row = box + Y * RS + 1 + (X >> 5);
    return __funnelshift_r(row[0], row[1], X & 31) & 0x1ffu;
}

// The unit at smem `u` (NB bytes, any alignment) into the state box and its
// pattern into the mask box, at box unit position (bx, by).
template <int P, int Y>
__device__ __forceinline__ void tb_scatter_row(const uint32_t *v, uint32_t *box, uint32_t *mask, int RS, int bx, int by)
{
    const uint32_t xz[kFrame] = {};
    const uint32_t w0 = assemble<RowWord<P, Y + 1, 0>>(v, xz, nullptr);
    const uint32_t w1 = assemble<RowWord<P, Y + 1, 1>>(v, xz, nullptr);
    const uint32_t w2 = assemble<RowWord<P, Y + 1, 2>>(v, xz, nullptr);
    const uint32_t bits = (tb_nibble(w0) >> 1) | (tb_nibble(w1) << 3) | ((tb_nibble(w2) & 3u) << 7);
    if (bits) tb_or_bits(box, RS, 9 * by + Y, 9 * bx, bits);
    tb_or_bits(mask, RS, 9 * by + Y, 9 * bx, tb_pattern<P>(Y));
}

template <int P, int... Y>
__device__ __forceinline__ void tb_scatter_unit(const uint8_t *u, uint32_t *box, uint32_t *mask, int RS, int bx, int by,
                                                std::integer_sequence<int, Y...>)
{
    constexpr int NB = RowsPreset<P>::k * RowsPreset<P>::k, NW = (NB + 3) / 4;
    const uint8_t *wp = reinterpret_cast<const uint8_t *>((uintptr_t)u & ~(uintptr_t)3);
    const uint32_t sh = (uint32_t)((uintptr_t)u & 3) * 8u;
    uint32_t v[NW];
    {
        uint32_t w[NW + 1];
#pragma unroll
        for (int i = 0; i <= NW; ++i) w[i] = lds32(wp + 4 * i);
#pragma unroll
        for (int i = 0; i < NW; ++i) v[i] = bytes_to_01(__funnelshift_r(w[i], w[i + 1], sh));
        if constexpr (NB % 4) v[NW - 1] &= 0xffffffffu >> (8 * (4 - NB % 4));
    }
    (tb_scatter_row<P, Y>(v, box, mask, RS, bx, by), ...);
}

template <int P, int... I>
__device__ __forceinline__ void tb_gather_words(const uint32_t *t, uint32_t *o, std::integer_sequence<int, I...>)
{
    ((o[I] = assemble<TotalWord<P, I>>(nullptr, nullptr, t)), ...);
}

// One generation of a box word from the words of its row and the rows
// above (a) and below (e), each with its west (_m) and east (_p) neighbour
// words: Life-like rule over the 8 Moore neighbours, bit-sliced, masked.
// LIFE: the rule is B3/S23 (new = count is 3, or 2 and alive); otherwise
// tb / ts hold the birth / survival tables for counts 0..8 as all-ones or
// zero words.
template <bool LIFE>
__device__ __forceinline__ uint32_t tb_cell_word(uint32_t a_m, uint32_t a, uint32_t a_p, uint32_t c_m, uint32_t c,
                                                 uint32_t c_p, uint32_t e_m, uint32_t e, uint32_t e_p, uint32_t m,
                                                 const uint32_t *tb, const uint32_t *ts)
{
    const uint32_t aW = __funnelshift_l(a_m, a, 1), aE = __funnelshift_r(a, a_p, 1);
    const uint32_t cW = __funnelshift_l(c_m, c, 1), cE = __funnelshift_r(c, c_p, 1);
    const uint32_t eW = __funnelshift_l(e_m, e, 1), eE = __funnelshift_r(e, e_p, 1);
    // 8-input adder: count = 8 b3 + 4 b2 + 2 b1 + b0
    const uint32_t s0 = aW ^ a ^ aE, k0 = (aW & a) | (aE & (aW ^ a));
    const uint32_t s1 = cW ^ cE ^ eW, k1 = (cW & cE) | (eW & (cW ^ cE));
    const uint32_t s2 = e ^ eE, k2 = e & eE;
    const uint32_t b0 = s0 ^ s1 ^ s2, k3 = (s0 & s1) | (s2 & (s0 ^ s1));
    const uint32_t t0 = k0 ^ k1 ^ k2, d0 = (k0 & k1) | (k2 & (k0 ^ k1));
    const uint32_t b1 = t0 ^ k3, d1 = t0 & k3;
    if constexpr (LIFE) {
        // count 2 or 3 (b1 set, no 4 or 8), and b0 or alive: d0 | d1 is 4 or 8
        return b1 & ~(d0 | d1) & (b0 | c) & m;
    } else {
        const uint32_t b2 = d0 ^ d1, b3 = d0 & d1;
        const uint32_t nb = tb_sel(b3, tb[8],
                                   tb_sel(b2, tb_sel(b1, tb_sel(b0, tb[7], tb[6]), tb_sel(b0, tb[5], tb[4])),
                                          tb_sel(b1, tb_sel(b0, tb[3], tb[2]), tb_sel(b0, tb[1], tb[0]))));
        const uint32_t ns = tb_sel(b3, ts[8],
                                   tb_sel(b2, tb_sel(b1, tb_sel(b0, ts[7], ts[6]), tb_sel(b0, ts[5], ts[4])),
                                          tb_sel(b1, tb_sel(b0, ts[3], ts[2]), tb_sel(b0, ts[1], ts[0]))));
        return tb_sel(c, ns, nb) & m;
    }
}

template <int P, bool LIFE>
__global__ void __launch_bounds__(256) step_tb_kernel(TbArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    constexpr int NB = RowsPreset<P>::k * RowsPreset<P>::k, NW = (NB + 3) / 4;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *tile = smem;
    uint8_t *halo = smem + a.off_halo;
    uint8_t *pres = smem + a.off_pres;
    uint32_t *box0 = reinterpret_cast<uint32_t *>(smem + a.off_box0);
    uint32_t *box1 = reinterpret_cast<uint32_t *>(smem + a.off_box1);
    uint32_t *mask = reinterpret_cast<uint32_t *>(smem + a.off_mask);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int boxw = a.W * a.RS;
    uint32_t tbl[9], tsl[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        tbl[j] = ((a.birth >> j) & 1u) ? 0xffffffffu : 0u;
        tsl[j] = ((a.survive >> j) & 1u) ? 0xffffffffu : 0u;
    }
    for (int i = tid; i < boxw; i += nth) box1[i] = 0;   // its guard words stay 0
    const int nstrip = nth / a.NWB;                     // strips of rows per word column
    const int my_strip = tid / a.NWB, my_w = 1 + tid % a.NWB;
    for (int64_t T = blockIdx.x; T < a.NT; T += gridDim.x) {
        // 1. the tile's bytes and the present halo units, into shared memory;
        // the state and mask boxes cleared
        const uint8_t *src = in + T * a.KL;
        if ((((uintptr_t)src) & 15) == 0 && (a.KL & 15) == 0) {
            for (int64_t i = tid; i < a.KL / 16; i += nth)
                reinterpret_cast<uint4 *>(tile)[i] = reinterpret_cast<const uint4 *>(src)[i];
        } else {
            for (int64_t i = tid; i < a.KL; i += nth) tile[i] = src[i];
        }
        for (int e = tid; e < a.nring; e += nth) {
            const uint32_t w = __ldg(a.ring + 2 * e);
            const int32_t tn = __ldg(a.nbr + T * 8 + (w >> 24));
            pres[e] = tn >= 0;
            if (tn >= 0) {
                const uint8_t *hs = in + (int64_t)tn * a.KL + (int64_t)NB * (w & 0xffffffu);
                uint8_t *hd = halo + NB * e;
                if ((NB & 15) == 0 && (((uintptr_t)hs) & 15) == 0) {
#pragma unroll
                    for (int i = 0; i < NB / 16; ++i)
                        reinterpret_cast<uint4 *>(hd)[i] = reinterpret_cast<const uint4 *>(hs)[i];
                } else {
                    for (int i = 0; i < NB; ++i) hd[i] = hs[i];
                }
            }
        }
        for (int i = tid; i < boxw; i += nth) {
            box0[i] = 0;
            mask[i] = 0;
        }
        __syncthreads();
        // 2. units into the boxes
        for (int q = tid; q < a.nu + a.nring; q += nth) {
            int bx, by;
            const uint8_t *u;
            if (q < a.nu) {
                const uint32_t p = __ldg(a.upos + q);
                bx = p & 0xff;
                by = p >> 8;
                u = tile + NB * q;
            } else {
                const int e = q - a.nu;
                if (!pres[e]) continue;
                const uint32_t p = __ldg(a.ring + 2 * e + 1);
                bx = p & 0xff;
                by = p >> 8;
                u = halo + NB * e;
            }
            tb_scatter_unit<P>(u, box0, mask, a.RS, bx, by, std::make_integer_sequence<int, 9>());
        }
        __syncthreads();
        // 3. the generations, each over the rows it can still compute
        // exactly: thread (strip, w) walks down word column w of its strip of
        // rows, keeping three rows of three words in registers
        uint32_t *cur = box0, *nxt = box1;
        for (int j = 1; j <= a.gens; ++j) {
            const int rows = a.W - 2 * j;
            const int len = (rows + nstrip - 1) / nstrip;
            const int y0 = j + my_strip * len, y1 = min(y0 + len, a.W - j);
            if (my_strip < nstrip && y0 < y1) {
                const uint32_t *sp = cur + (y0 - 1) * a.RS + my_w;
                uint32_t a_m = sp[-1], a0 = sp[0], a_p = sp[1];
                sp += a.RS;
                uint32_t c_m = sp[-1], c0 = sp[0], c_p = sp[1];
                for (int y = y0; y < y1; ++y) {
                    sp += a.RS;
                    const uint32_t e_m = sp[-1], e0 = sp[0], e_p = sp[1];
                    const int at = y * a.RS + my_w;
                    nxt[at] = tb_cell_word<LIFE>(a_m, a0, a_p, c_m, c0, c_p, e_m, e0, e_p, mask[at], tbl, tsl);
                    a_m = c_m; a0 = c0; a_p = c_p;
                    c_m = e_m; c0 = e0; c_p = e_p;
                }
            }
            __syncthreads();
            uint32_t *t = cur;
            cur = nxt;
            nxt = t;
        }
        // 4. the tile's units back to omega order
        uint8_t *dst = out + T * a.KL;
        for (int q = tid; q < a.nu; q += nth) {
            const uint32_t p = __ldg(a.upos + q);
            const int bx = p & 0xff, by = p >> 8;
            uint32_t t[27];
#pragma unroll
            for (int y = 0; y < 9; ++y) {
                const uint32_t bits = tb_get_bits(cur, a.RS, 9 * by + y, 9 * bx);
                t[3 * y] = tb_expand4(bits & 15u);
                t[3 * y + 1] = tb_expand4((bits >> 4) & 15u);
                t[3 * y + 2] = ((bits >> 8) & 1u) << 16;
            }
            uint32_t o[NW];
            tb_gather_words<P>(t, o, std::make_integer_sequence<int, NW>());
            uint8_t *ud = dst + (int64_t)NB * q;
            if ((NB & 15) == 0 && (((uintptr_t)ud) & 15) == 0) {
#pragma unroll
                for (int i = 0; i < NW / 4; ++i)
                    reinterpret_cast<uint4 *>(ud)[i] = make_uint4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < NB; ++i) ud[i] = (uint8_t)(o[i / 4] >> (8 * (i % 4)));
            }
        }
        __syncthreads();   // shared memory is reused by the next tile
    }
}

}  // namespace fr
