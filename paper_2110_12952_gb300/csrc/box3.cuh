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
// totals.  Box offsets of the tile's cells are 16-bit, two per table word,
// read from global memory (the same for every tile, so they stay in L1);
// results go straight to memory.  Without a table or an output stage in
// shared memory a tile of depth 3 needs 70 KB: three blocks per SM.
#pragma once

#include <stdint.h>

namespace fr {

// Totals of the interior box rows (1 <= y, z <= B), NC 16-byte chunks per
// row.  A team of TEAM >= NC consecutive lanes takes the rows y0 .. y0 +
// S - 1 of plane z, lane c of it chunk c (so that the 8 lanes of a
// quarter-warp read 8 different 16-byte bank groups).  Sliding down y, each
// lane keeps the plane sums P(y) = row(y, z - 1) + row(y, z) + row(y, z +
// 1) of its chunk for three rows, so that the column sums V(y) = P(y - 1) +
// P(y) + P(y + 1) (<= 9 per byte) cost three row loads each; it gets the
// last column sum of chunk c - 1 and the first of chunk c + 1 from its team
// neighbours and forms for box position 4w + j the sum of column sums
// 4w + j - 1 .. 4w + j + 1 with funnel shifts (<= 27 per byte: no carries).
template <int NC, int TEAM, int S>
__device__ __forceinline__ void box3_rows(const StepArgs &a, const uint8_t *box, uint8_t *tbox)
{
    const int B = a.Py - 2, Px = a.Px, PxPy = a.Px * a.Py, nseg = (B + S - 1) / S, items = B * nseg;
    const int tid = threadIdx.x, c = tid % TEAM;
    for (int i0 = 0; i0 < items; i0 += (int)blockDim.x / TEAM) {
        const int it = i0 + tid / TEAM;
        const bool lane_ok = it < items && c < NC;
        const int z = 1 + it % B, y0 = 1 + S * (it / B);
        // byte offset of (y0, z), chunk c; only rows y <= B are stored
        const int base = lane_ok ? Px * y0 + PxPy * z + 16 * c : 0;
        auto plane_sum = [&](int dy, uint32_t *P) {
            P[0] = P[1] = P[2] = P[3] = 0u;
            if (lane_ok && y0 + dy <= B + 1) {   // rows past the box only feed rows past B
#pragma unroll
                for (int dz = -1; dz <= 1; ++dz) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(box + base + dy * Px + dz * PxPy);
                    P[0] += q.x;
                    P[1] += q.y;
                    P[2] += q.z;
                    P[3] += q.w;
                }
            }
        };
        uint32_t Pa[4], Pb[4];
        plane_sum(-1, Pa);
        plane_sum(0, Pb);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            uint32_t Pc[4];
            plane_sum(k + 1, Pc);
            uint32_t V[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) V[w] = Pa[w] + Pb[w] + Pc[w];
            uint32_t prev = 0u, next = 0u;
            if constexpr (TEAM > 1) {
                prev = __shfl_up_sync(0xffffffffu, V[3], 1, TEAM);
                next = __shfl_down_sync(0xffffffffu, V[0], 1, TEAM);
                if (c == 0) prev = 0u;
                if (c + 1 >= NC) next = 0u;
            }
            if (lane_ok && y0 + k <= B) {
                uint32_t T[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const uint32_t lo = (w > 0) ? V[w - 1] : prev, hi = (w < 3) ? V[w + 1] : next;
                    T[w] = __funnelshift_r(lo, V[w], 24) + V[w] + __funnelshift_r(V[w], hi, 8);
                }
                *reinterpret_cast<uint4 *>(tbox + base + k * Px) = make_uint4(T[0], T[1], T[2], T[3]);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                Pa[w] = Pb[w];
                Pb[w] = Pc[w];
            }
        }
    }
}

struct Box3Policy {
    static constexpr bool kRingInTile = false;   // halo bytes go to the box
    static constexpr bool kDirectStore = true;   // no output stage
    struct Regs {};
    __device__ static void init(const StepArgs &, Regs &) {}
    // four consecutive cells per thread: their box offsets in one 8-byte
    // load, their states from two aligned words of the input stage
    __device__ static void scatter(const StepArgs &a, const TileIO &io, uint8_t *box, const uint32_t *, Regs &)
    {
        const uint2 *tab4 = reinterpret_cast<const uint2 *>(a.tab);   // 4 offsets per entry
        const uint8_t *wp = io.data + (io.a_in & ~3);
        const uint32_t sh = 8u * (uint32_t)(io.a_in & 3);
        for (int64_t l0 = 4 * (int64_t)threadIdx.x; l0 < a.KL; l0 += 4 * (int64_t)blockDim.x) {
            const uint2 pp = __ldg(tab4 + l0 / 4);
            const uint32_t p[4] = {pp.x & 0xffffu, pp.x >> 16, pp.y & 0xffffu, pp.y >> 16};
            const uint32_t st = __funnelshift_r(lds32(wp + l0), lds32(wp + l0 + 4), sh);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (l0 + i < a.KL) box[p[i]] = ((st >> (8 * i)) & 0xffu) != 0;
        }
    }
    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *box, const uint32_t *,
                                   Regs &)
    {
        uint8_t *tbox = const_cast<uint8_t *>(box) + a.box_bytes / 2;
        switch (a.Px >> 4) {
            case 1: box3_rows<1, 1, 3>(a, box, tbox); break;
            case 2: box3_rows<2, 2, 3>(a, box, tbox); break;
            case 3: box3_rows<3, 4, 3>(a, box, tbox); break;
            default: box3_rows<4, 4, 3>(a, box, tbox); break;
        }
        __syncthreads();
        // four consecutive cells per thread: their box offsets in one 8-byte
        // load, state and total from the two boxes (the input stage is being
        // refilled by now); a live cell's total counts itself, hence the
        // survival mask shifted up by one.  The four results go to memory as
        // one word where it is aligned (a warp writes 128 consecutive bytes)
        const uint2 *tab4 = reinterpret_cast<const uint2 *>(a.tab);
        const uint32_t live = io.rule.survive << 1, dead = io.rule.birth;
        for (int64_t l0 = 4 * (int64_t)threadIdx.x; l0 < a.KL; l0 += 4 * (int64_t)blockDim.x) {
            const uint2 pp = __ldg(tab4 + l0 / 4);
            const uint32_t p[4] = {pp.x & 0xffffu, pp.x >> 16, pp.y & 0xffffu, pp.y >> 16};
            uint32_t w = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (l0 + i < a.KL) w |= (((box[p[i]] ? live : dead) >> tbox[p[i]]) & 1u) << (8 * i);
            uint8_t *op = io.gout + l0;
            if (l0 + 4 <= a.KL && ((uintptr_t)op & 3) == 0) {
                *reinterpret_cast<uint32_t *>(op) = w;
            } else {
                for (int i = 0; i < 4 && l0 + i < a.KL; ++i) op[i] = (uint8_t)(w >> (8 * i));
            }
        }
    }
};

}  // namespace fr
