// box3.cuh -- device side of the "box3" policy of the compact step for 3D
// fractals (the Menger sponge): the tile sits in its padded box as in the
// cell policy, but the 27-cell totals of the 26-neighbour rule (Sec. 3
// stencil, extended to three dimensions) are formed for whole box rows at
// once, four cells per 32-bit word (phase A); each member cell then gathers
// its own total in omega order and applies the rule (phase B).  Included by
// step.cu after its device helpers.
//
// Box layout (host plan): rows of Px bytes (a multiple of 16 with at least
// one zero word after the last padded cell), Py = B + 2 rows per plane,
// B + 2 planes; a second box of the same layout right after it holds the
// totals.  Box offsets of the tile's cells are 16-bit, two per table word.
#pragma once

#include <stdint.h>

namespace fr {

// Totals of the box row at byte offset `off` (an interior row: 1 <= y, z <=
// B): the column sums over the 9 rows (y + dy, z + dz) in NWR words, then
// for box position 4w + j the sum of columns 4w + j - 1 .. 4w + j + 1 from
// words w - 1, w, w + 1 with funnel shifts.  Bytes stay <= 27: no carries.
template <int NWR>
__device__ __forceinline__ void box3_row(const uint8_t *box, uint8_t *tbox, int off, int Px, int PxPy)
{
    uint32_t V[NWR];
#pragma unroll
    for (int w = 0; w < NWR; ++w) V[w] = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const uint4 *rp = reinterpret_cast<const uint4 *>(box + off + dy * Px + dz * PxPy);
#pragma unroll
            for (int c = 0; c < NWR / 4; ++c) {
                const uint4 q = rp[c];
                V[4 * c] += q.x;
                V[4 * c + 1] += q.y;
                V[4 * c + 2] += q.z;
                V[4 * c + 3] += q.w;
            }
        }
    uint4 *tp = reinterpret_cast<uint4 *>(tbox + off);
#pragma unroll
    for (int c = 0; c < NWR / 4; ++c) {
        uint32_t T[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int w = 4 * c + j;
            const uint32_t prev = (w > 0) ? V[w - 1] : 0u, next = (w + 1 < NWR) ? V[w + 1] : 0u;
            T[j] = __funnelshift_r(prev, V[w], 24) + V[w] + __funnelshift_r(V[w], next, 8);
        }
        tp[c] = make_uint4(T[0], T[1], T[2], T[3]);
    }
}

template <int NWR>
__device__ __forceinline__ void box3_rows(const StepArgs &a, const uint8_t *box, uint8_t *tbox)
{
    const int B = a.Py - 2, Px = a.Px, PxPy = a.Px * a.Py;
    for (int i = threadIdx.x; i < B * B; i += blockDim.x) {
        const int y = 1 + i % B, z = 1 + i / B;
        box3_row<NWR>(box, tbox, Px * y + PxPy * z, Px, PxPy);
    }
}

struct Box3Policy {
    static constexpr bool kRingInTile = false;   // halo bytes go to the box
    struct Regs {};
    __device__ static void init(const StepArgs &, Regs &) {}
    __device__ static void scatter(const StepArgs &a, const TileIO &io, uint8_t *box, const uint32_t *tab, Regs &)
    {
        const uint16_t *tab16 = reinterpret_cast<const uint16_t *>(tab);
        const uint8_t *tin = io.data + io.a_in;
        for (int64_t l = threadIdx.x; l < a.KL; l += blockDim.x) box[tab16[l]] = tin[l] != 0;
    }
    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *box, const uint32_t *tab,
                                   Regs &)
    {
        uint8_t *tbox = const_cast<uint8_t *>(box) + a.box_bytes / 2;
        switch (a.Px >> 2) {
            case 4: box3_rows<4>(a, box, tbox); break;
            case 8: box3_rows<8>(a, box, tbox); break;
            case 12: box3_rows<12>(a, box, tbox); break;
            default: box3_rows<16>(a, box, tbox); break;
        }
        __syncthreads();
        // four consecutive cells per thread: their box offsets in one 8-byte
        // load, total and state from the boxes; a live cell's total counts
        // itself, hence the survival mask shifted up by one
        const uint16_t *tab16 = reinterpret_cast<const uint16_t *>(tab);
        uint8_t *tout = io.ostage + io.a_out;
        const uint32_t live = io.rule.survive << 1, dead = io.rule.birth;
        for (int64_t l0 = 4 * (int64_t)threadIdx.x; l0 < a.KL; l0 += 4 * (int64_t)blockDim.x) {
            const uint2 pp = *reinterpret_cast<const uint2 *>(tab16 + l0);
            const uint32_t p[4] = {pp.x & 0xffffu, pp.x >> 16, pp.y & 0xffffu, pp.y >> 16};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (l0 + i < a.KL) tout[l0 + i] = (uint8_t)(((box[p[i]] ? live : dead) >> tbox[p[i]]) & 1u);
        }
    }
};

}  // namespace fr
