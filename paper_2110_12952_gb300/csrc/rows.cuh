// rows.cuh -- device side of the "rows" policy of the compact step (see
// rows_layout.h for the unit layout): compile-time word assembly with prmt,
// and the policy itself.  Included by step.cu after its device helpers.
#pragma once

#include <stdint.h>

#include <utility>

#include "rows_layout.h"

namespace fr {

// ---- compile-time word assembly: a word whose byte i is byte b_i of one of
// up to four registers (or zero), with one, two or three prmt.
//   kind 0: a state word (bytes 0 or 1; prmt's sign mode on it gives 0)
//   kind 1: a zero-extended byte (bytes 1..3 are 0)
//   kind 2: a totals word (no zero byte; "zero" means "don't care" there)
struct Src {
    int kind, reg, byte;   // kind -1: zero
};
struct WordPlan {
    int n;
    int kind[4], reg[4];
    uint32_t s1, s2, s3;   // selectors: (r0, r1), then (r2, r3) or (result, r2), then (a, b)
};

constexpr int reg_index(const WordPlan &p, const Src &s)
{
    for (int i = 0; i < p.n; ++i)
        if (p.kind[i] == s.kind && p.reg[i] == s.reg) return i;
    return -1;
}

// selector nibble of a zero byte from the pair (a, b)
constexpr uint32_t zero_nibble(int kind_a, int kind_b)
{
    if (kind_b == 1) return 5;        // byte 1 of a zero-extended b
    if (kind_a == 1) return 1;        // byte 1 of a zero-extended a
    if (kind_b == 0) return 0xC;      // sign of b's byte 0 (0 or 1)
    if (kind_a == 0) return 0x8;      // sign of a's byte 0
    return 0;                         // don't care
}

constexpr WordPlan plan_word(Src s0, Src s1, Src s2, Src s3)
{
    WordPlan p{0, {0, 0, 0, 0}, {0, 0, 0, 0}, 0u, 0u, 0u};
    const Src s[4] = {s0, s1, s2, s3};
    for (int i = 0; i < 4; ++i) {
        if (s[i].kind < 0) continue;
        if (reg_index(p, s[i]) < 0) {
            p.kind[p.n] = s[i].kind;
            p.reg[p.n] = s[i].reg;
            ++p.n;
        }
    }
    uint32_t a = 0, b = 0, c = 0;
    for (int i = 0; i < 4; ++i) {
        const int r = s[i].kind < 0 ? -1 : reg_index(p, s[i]);
        uint32_t na = 0, nb = 0, nc = 0;
        if (p.n <= 2) {
            if (r == 0) na = (uint32_t)s[i].byte;
            else if (r == 1) na = 4u + (uint32_t)s[i].byte;
            else na = (p.n == 1) ? (p.kind[0] == 2 ? 0u : 4u) : zero_nibble(p.kind[0], p.kind[1]);
        } else if (p.n == 3) {
            na = (r == 0) ? (uint32_t)s[i].byte : (r == 1 ? 4u + (uint32_t)s[i].byte : 0u);
            if (r == 0 || r == 1) nb = (uint32_t)i;
            else if (r == 2) nb = 4u + (uint32_t)s[i].byte;
            else nb = (p.kind[2] == 1) ? 5u : (p.kind[2] == 0 ? 0xCu : (uint32_t)i);
        } else {
            na = (r == 0) ? (uint32_t)s[i].byte : (r == 1 ? 4u + (uint32_t)s[i].byte : 0u);
            nb = (r == 2) ? (uint32_t)s[i].byte : (r == 3 ? 4u + (uint32_t)s[i].byte : 0u);
            if (r == 2 || r == 3) nc = 4u + (uint32_t)i;
            else if (r == 0 || r == 1) nc = (uint32_t)i;
            else nc = 0u;   // with four registers every byte has a source
        }
        a |= na << (4 * i);
        b |= nb << (4 * i);
        c |= nc << (4 * i);
    }
    p.s1 = a;
    p.s2 = b;
    p.s3 = c;
    return p;
}

template <int K, int R>
__device__ __forceinline__ uint32_t pick(const uint32_t *v, const uint32_t *x, const uint32_t *t)
{
    if constexpr (K == 0) return v[R];
    else if constexpr (K == 1) return x[R];
    else return t[R];
}

template <class Gen>
__device__ __forceinline__ uint32_t assemble(const uint32_t *v, const uint32_t *x, const uint32_t *t)
{
    constexpr WordPlan p = Gen::plan();
    if constexpr (p.n == 0) {
        return 0u;
    } else if constexpr (p.n == 1) {
        if constexpr (p.s1 == 0x3210u) return pick<p.kind[0], p.reg[0]>(v, x, t);
        else return prmt(pick<p.kind[0], p.reg[0]>(v, x, t), 0u, p.s1);
    } else if constexpr (p.n == 2) {
        return prmt(pick<p.kind[0], p.reg[0]>(v, x, t), pick<p.kind[1], p.reg[1]>(v, x, t), p.s1);
    } else if constexpr (p.n == 3) {
        const uint32_t ab = prmt(pick<p.kind[0], p.reg[0]>(v, x, t), pick<p.kind[1], p.reg[1]>(v, x, t), p.s1);
        return prmt(ab, pick<p.kind[2], p.reg[2]>(v, x, t), p.s2);
    } else {
        const uint32_t ab = prmt(pick<p.kind[0], p.reg[0]>(v, x, t), pick<p.kind[1], p.reg[1]>(v, x, t), p.s1);
        const uint32_t cd = prmt(pick<p.kind[2], p.reg[2]>(v, x, t), pick<p.kind[3], p.reg[3]>(v, x, t), p.s2);
        return prmt(ab, cd, p.s3);
    }
}

// Row RY (= y + 1, y = -1..9) word W (columns 4W - 1 .. 4W + 2) of the
// unit's window: own cells from the state words v, frame cells from the
// zero-extended external bytes x, zeros for holes and column 10.
template <int P>
constexpr Src row_src(int ry, int w, int b)
{
    const int x = 4 * w + b - 1, y = ry - 1;
    if (x >= 0 && x <= 8 && y >= 0 && y <= 8) {
        const int u = rp_byte<P>(x, y);
        return u < 0 ? Src{-1, 0, 0} : Src{0, u / 4, u % 4};
    }
    const int t = frame_at(x, y);
    if (t < 0) return Src{-1, 0, 0};
    const int e = ext_of_frame<P>(t);
    return e < 0 ? Src{-1, 0, 0} : Src{1, e, 0};
}
template <int P, int RY, int W>
struct RowWord {
    static constexpr WordPlan plan()
    {
        return plan_word(row_src<P>(RY, W, 0), row_src<P>(RY, W, 1), row_src<P>(RY, W, 2), row_src<P>(RY, W, 3));
    }
};

// Totals row y: t[3y] = columns 0..3, t[3y + 1] = 4..7, byte 2 of t[3y + 2] =
// column 8.  Omega word I of the unit gathers its 4 cells' totals.
template <int P>
constexpr Src total_src(int u)
{
    if (u >= RowsPreset<P>::k * RowsPreset<P>::k) return Src{-1, 0, 0};
    const int x = rp_x<P>(u), y = rp_y<P>(u);
    return x < 8 ? Src{2, 3 * y + x / 4, x % 4} : Src{2, 3 * y + 2, 2};
}
template <int P, int I>
struct TotalWord {
    static constexpr WordPlan plan()
    {
        return plan_word(total_src<P>(4 * I), total_src<P>(4 * I + 1), total_src<P>(4 * I + 2),
                         total_src<P>(4 * I + 3));
    }
};

template <int P, int E>
__device__ __forceinline__ uint32_t rows_ext(const uint8_t *tin, const uint32_t *e)
{
    constexpr int t = frame_of_ext<P>(E);
    constexpr int d = frame_dir(t), b = frame_byte<P>(t);
    return min((uint32_t)tin[e[d] + b], 1u);
}

// The work of a unit in three bands of three rows (Y = 0..2): band Y
// loads the frame cells of the rows it adds, builds those rows (window rows
// 3Y + 2 .. 3Y + 4, and rows 0, 1 as well for Y = 0), sums totals rows 3Y ..
// 3Y + 2, and gathers and rules the omega words whose cells lie in rows up
// to 3Y + 2, so that few values are live at once.
template <int P>
constexpr int ext_row(int e) { return frame_y(frame_of_ext<P>(e)) + 1; }
template <int P>
constexpr int word_band(int i)
{
    int band = 0;
    for (int b = 0; b < 4; ++b) {
        const int u = 4 * i + b;
        if (u < RowsPreset<P>::k * RowsPreset<P>::k && rp_y<P>(u) / 3 > band) band = rp_y<P>(u) / 3;
    }
    return band;
}

template <int P, int Y, int E>
__device__ __forceinline__ void band_ext(const uint8_t *tin, const uint32_t *e, uint32_t *x)
{
    constexpr int ry = ext_row<P>(E), lo = (Y == 0) ? 0 : 3 * Y + 2;
    if constexpr (ry >= lo && ry <= 3 * Y + 4) x[E] = rows_ext<P, E>(tin, e);
}
template <int P, int Y, int RY>
__device__ __forceinline__ void band_row(const uint32_t *v, const uint32_t *x, uint32_t *r)
{
    constexpr int lo = (Y == 0) ? 0 : 3 * Y + 2;
    if constexpr (RY >= lo && RY <= 3 * Y + 4) {
        r[3 * RY] = assemble<RowWord<P, RY, 0>>(v, x, nullptr);
        r[3 * RY + 1] = assemble<RowWord<P, RY, 1>>(v, x, nullptr);
        r[3 * RY + 2] = assemble<RowWord<P, RY, 2>>(v, x, nullptr);
    }
}
template <int P, int Y, int I>
__device__ __forceinline__ void band_word(const Rule &rule, const uint32_t *v, const uint32_t *t, uint32_t *o)
{
    if constexpr (word_band<P>(I) == Y) o[I] = rule4(rule.lut, assemble<TotalWord<P, I>>(nullptr, nullptr, t), v[I]);
}
template <int P, int Y, int... E, int... RY, int... I>
__device__ __forceinline__ void unit_band(const uint8_t *tin, const uint32_t *e, const Rule &rule, const uint32_t *v,
                                          uint32_t *x, uint32_t *r, uint32_t *t, uint32_t *o,
                                          std::integer_sequence<int, E...>, std::integer_sequence<int, RY...>,
                                          std::integer_sequence<int, I...>)
{
    (band_ext<P, Y, E>(tin, e, x), ...);
    (band_row<P, Y, RY>(v, x, r), ...);
#pragma unroll
    for (int y = 3 * Y; y < 3 * Y + 3; ++y) {
        // additions as integer multiply-adds by kOne: the FMA pipe, not the ALU
        const uint32_t one = kOne;
        const uint32_t V0 = mad_u32(mad_u32(r[3 * y], one, r[3 * y + 3]), one, r[3 * y + 6]);
        const uint32_t V1 = mad_u32(mad_u32(r[3 * y + 1], one, r[3 * y + 4]), one, r[3 * y + 7]);
        const uint32_t V2 = mad_u32(mad_u32(r[3 * y + 2], one, r[3 * y + 5]), one, r[3 * y + 8]);
        t[3 * y] = mad_u32(mad_u32(V0, one, __funnelshift_r(V0, V1, 8)), one, __funnelshift_r(V0, V1, 16));
        t[3 * y + 1] = mad_u32(mad_u32(V1, one, __funnelshift_r(V1, V2, 8)), one, __funnelshift_r(V1, V2, 16));
        t[3 * y + 2] = V2 * 0x010101u;
    }
    (band_word<P, Y, I>(rule, v, t, o), ...);
}

// Bytes 0..NB-1 of unit q (NB bytes per unit, contiguous in the stage) as
// words v[0..NW-1], cells 0 or 1 (bytes past the unit: whatever follows).
template <int NB, int NW>
__device__ __forceinline__ void load_unit(const TileIO &io, int q, uint32_t *v)
{
    constexpr uint32_t kLastMask = (NB % 4) ? (0xffffffffu >> (8 * (4 - NB % 4))) : 0xffffffffu;
    const int off = io.a_in + NB * q;
    const uint8_t *wp = io.data + (off & ~3);
    const uint32_t sh = (uint32_t)(off & 3) * 8u;
    uint32_t w[NW + 1];
#pragma unroll
    for (int i = 0; i <= NW; ++i) w[i] = lds32(wp + 4 * i);
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        v[i] = __funnelshift_r(w[i], w[i + 1], sh);
        any |= (i == NW - 1) ? (v[i] & kLastMask) : v[i];
    }
    if (any & 0xfefefefeu) {
#pragma unroll
        for (int i = 0; i < NW; ++i) v[i] = bytes_to_01(v[i]);
    }
}

// Bytes 0..NB-1 of o to unit q of the output stage: word i of the aligned run
// from the unit's first byte - m holds bytes 4i - m .. 4i - m + 3; words
// holding only this unit's bytes are stored whole, the others byte by byte.
// o has NW + 1 words, o[NW] = 0.
template <int NB, int NW>
__device__ __forceinline__ void store_unit(const TileIO &io, int q, const uint32_t *o)
{
    uint8_t *ob = io.ostage + io.a_out + NB * q;
    const uint32_t m = (uint32_t)(io.a_out + NB * q) & 3u;
    uint8_t *base = ob - m;
    const uint32_t sl = 8u * m;
#pragma unroll
    for (int i = 0; i <= NW; ++i) {
        const uint32_t wv = (i == 0) ? (o[0] << sl) : __funnelshift_l(o[i - 1], o[i], sl);
        if (4 * i >= 3 && 4 * i + 4 <= NB) {
            sts32(base + 4 * i, wv);
        } else {
            const int lo = 4 * i - (int)m;   // byte of the unit at the word's byte 0
            if (lo >= 0 && lo + 4 <= NB) {
                sts32(base + 4 * i, wv);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (lo + j >= 0 && lo + j < NB) base[4 * i + j] = (uint8_t)(wv >> (8 * j));
            }
        }
    }
}

template <int P>
struct RowsPolicy {
    static constexpr bool kRingInTile = true;   // halo units go after the tile's bytes
    static constexpr int K = RowsPreset<P>::k;
    static constexpr int NB = K * K;            // bytes per unit
    static constexpr int NW = (NB + 3) / 4;     // words per unit
    static constexpr int NE = rp_next<P>();     // external cells per unit
    // units in their own slots of the stages (rp_slot), else the tile's
    // bytes as one copy
    static constexpr bool kPadded = rp_padded<P>();
    __host__ __device__ static constexpr int slot(int n) { return rp_slot<P>(n); }
    static constexpr bool kRingByAll = true;    // hundreds of halo cells per tile: every thread helps
    struct Regs {
        uint32_t e[8];   // byte offsets of the 8 neighbouring units (W..E, N..S)
    };
    static constexpr int kGroup = rp_group<P>();   // units per bulk copy of padded units
    static_assert(!kPadded || NB == 64, "padded units are 64 bytes");
    __device__ static void init(const StepArgs &a, Regs &R)
    {
        const int q = rp_thread_unit<P>(threadIdx.x, a.nq);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = (q < a.nq) ? __ldg(a.tab + 4 * q + k) : 0u;
            R.e[2 * k] = w & 0xffffu;
            R.e[2 * k + 1] = w >> 16;
        }
    }
    // the all-zero unit, after the halo units, by the lanes of the filling warp
    __device__ static void fill(const StepArgs &a, uint8_t *tin, int lane)
    {
        for (int j = lane; j < NB; j += 32) tin[slot(a.tapz) + j] = 0;
    }
    __device__ static void warp_bytes(const StepArgs &a, int w, int *b0, int *b1)
    {
        *b0 = NB * min(32 * w, a.nq);
        *b1 = NB * min(32 * w + 32, a.nq);
    }
    __device__ static void scatter(const StepArgs &, const TileIO &, uint8_t *, const uint32_t *, Regs &) {}

    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *, const uint32_t *,
                                   Regs &R)
    {
        if ((int)threadIdx.x >= a.nq) return;
        const int q = rp_thread_unit<P>(threadIdx.x, a.nq);
        uint32_t v[NW];
        uint32_t any = 0;
        if constexpr (kPadded) {
            // the unit sits 16-byte aligned at its own slot
            const uint8_t *up = io.data + slot(q);
#pragma unroll
            for (int c = 0; c < NW / 4; ++c) {
                const uint4 w4 = *reinterpret_cast<const uint4 *>(up + 16 * c);
                v[4 * c] = w4.x;
                v[4 * c + 1] = w4.y;
                v[4 * c + 2] = w4.z;
                v[4 * c + 3] = w4.w;
            }
#pragma unroll
            for (int i = 0; i < NW; ++i) any |= v[i];
            if (any & 0xfefefefeu) {
#pragma unroll
                for (int i = 0; i < NW; ++i) v[i] = bytes_to_01(v[i]);
            }
        } else {
            load_unit<NB, NW>(io, q, v);
        }
        const uint8_t *tin = kPadded ? io.data : io.data + io.a_in;
        uint32_t x[NE], r[33], t[27], o[NW + 1];
        unit_band<P, 0>(tin, R.e, io.rule, v, x, r, t, o, std::make_integer_sequence<int, NE>(),
                        std::make_integer_sequence<int, 11>(), std::make_integer_sequence<int, NW>());
        unit_band<P, 1>(tin, R.e, io.rule, v, x, r, t, o, std::make_integer_sequence<int, NE>(),
                        std::make_integer_sequence<int, 11>(), std::make_integer_sequence<int, NW>());
        unit_band<P, 2>(tin, R.e, io.rule, v, x, r, t, o, std::make_integer_sequence<int, NE>(),
                        std::make_integer_sequence<int, 11>(), std::make_integer_sequence<int, NW>());
        if constexpr (kPadded) {
            // the unit's 64 output bytes, 16-byte aligned in memory when the
            // buffer is
            uint8_t *op = io.gout + (int64_t)NB * q;
            if (((uintptr_t)op & 15) == 0) {
#pragma unroll
                for (int c = 0; c < NW / 4; ++c)
                    *reinterpret_cast<uint4 *>(op + 16 * c) = make_uint4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < NW; ++i)
                    for (int j = 0; j < 4; ++j) op[4 * i + j] = (uint8_t)(o[i] >> (8 * j));
            }
            return;
        }
        o[NW] = 0;
        store_unit<NB, NW>(io, q, o);
    }
};

}  // namespace fr
