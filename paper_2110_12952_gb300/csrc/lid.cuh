// lid.cuh -- device side of the "lid" policy of the compact step (see
// lid_layout.h for the unit layout).  Included by step.cu after rows.cuh,
// whose compile-time word assembly and unit load/store it uses.
#pragma once

#include <stdint.h>

#include <utility>

#include "lid_layout.h"
#include "rows.cuh"

namespace fr {

// Byte b of term word (W, direction D) of a unit: the neighbour in
// direction D (row-major over (dx, dy) in -1..1, D = 4 the cell itself) of
// unit byte 4W + b, from the unit's words, an external cell, or zero.
template <int P, int U>
constexpr Src lid_src(int w, int d, int b)
{
    const int u = 4 * w + b;
    if (u >= LidUnit<P, U>::NB) return Src{-1, 0, 0};
    const int x = lu_x<P, U>(u) + d % 3 - 1, y = lu_y<P, U>(u) + d / 3 - 1;
    const int n = lu_byte<P, U>(x, y);
    if (n >= 0) return Src{0, n / 4, n % 4};
    const int e = lu_ext_index<P, U>(x, y);
    return e >= 0 ? Src{1, e, 0} : Src{-1, 0, 0};
}
template <int P, int U, int W, int D>
struct LidTerm {
    static constexpr WordPlan plan()
    {
        return plan_word(lid_src<P, U>(W, D, 0), lid_src<P, U>(W, D, 1), lid_src<P, U>(W, D, 2),
                         lid_src<P, U>(W, D, 3));
    }
};

// totals of unit word W: the sum of its 9 term words (3x3 sums including the
// cell, <= 9 per byte: no carries), added as integer multiply-adds by kOne so
// that the additions issue on the FMA pipe rather than the ALU pipe, which
// the term words' prmt already keep busy
template <int P, int U, int W, int D>
__device__ __forceinline__ void lid_acc(const uint32_t *v, const uint32_t *x, uint32_t &t)
{
    if constexpr (D == 0) t = assemble<LidTerm<P, U, W, D>>(v, x, nullptr);
    else t = mad_u32(assemble<LidTerm<P, U, W, D>>(v, x, nullptr), kOne, t);
}
template <int P, int U, int W, int... D>
__device__ __forceinline__ uint32_t lid_total(const uint32_t *v, const uint32_t *x, std::integer_sequence<int, D...>)
{
    uint32_t t = 0;
    (lid_acc<P, U, W, D>(v, x, t), ...);
    return t;
}

template <int P, int U, int E>
__device__ __forceinline__ uint32_t lid_ext(const uint8_t *tin, const uint32_t *e)
{
    constexpr int x = lu_ext_x<P, U>(E), y = lu_ext_y<P, U>(E);
    constexpr int d = lu_dir<P, U>(x, y), b = lu_fbyte<P, U>(x, y);
    return min((uint32_t)tin[e[d] + b], 1u);
}

template <int P, int U, bool SPARSE, int... W>
__device__ __forceinline__ void lid_words(const Rule &rule, const uint32_t *v, const uint32_t *x, uint32_t *o,
                                          std::integer_sequence<int, W...>)
{
    if constexpr (SPARSE)
        ((o[W] = rule4_sparse(rule.lut_sparse, lid_total<P, U, W>(v, x, std::make_integer_sequence<int, 9>()), v[W])), ...);
    else
        ((o[W] = rule4(rule.lut, lid_total<P, U, W>(v, x, std::make_integer_sequence<int, 9>()), v[W])), ...);
}
template <int P, int U, int... E>
__device__ __forceinline__ void lid_exts(const uint8_t *tin, const uint32_t *e, uint32_t *x,
                                         std::integer_sequence<int, E...>)
{
    ((x[E] = lid_ext<P, U, E>(tin, e)), ...);
}

template <int P, int U>
struct LidPolicy {
    static constexpr bool kRingInTile = true;    // halo units go after the tile's bytes
    static constexpr bool kPadded = false;       // the tile's bytes as one copy
    __host__ __device__ static constexpr int slot(int n) { return LidUnit<P, U>::NB * n; }
    static constexpr bool kRingByAll = false;    // a few halo cells per tile
    static constexpr int NB = LidUnit<P, U>::NB;
    static constexpr int NW = (NB + 3) / 4;
    static constexpr int NE = lu_next<P, U>();
    static constexpr bool kSparse = lu_max_degree<P, U>() <= 6;   // t + 8 alive fits a nibble
    struct Regs {
        uint32_t e[8];   // byte offsets of the 8 neighbouring units
    };
    __device__ static void init(const StepArgs &a, Regs &R)
    {
        const int q = threadIdx.x;
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
        for (int j = lane; j < NB; j += 32) tin[NB * a.tapz + j] = 0;
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
        const int q = threadIdx.x;
        if (q >= a.nq) return;
        uint32_t v[NW], x[NE > 0 ? NE : 1], o[NW + 1];
        load_unit<NB, NW>(io, q, v);
        lid_exts<P, U>(io.data + io.a_in, R.e, x, std::make_integer_sequence<int, NE>());
        lid_words<P, U, kSparse>(io.rule, v, x, o, std::make_integer_sequence<int, NW>());
        o[NW] = 0;
        store_unit<NB, NW>(io, q, o);
    }
};

}  // namespace fr
