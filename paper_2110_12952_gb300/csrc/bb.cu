// bb.cu -- the bounding-box approach (Sec. 4, "BB"): the life-like rule on
// every cell of the n^dim box, the baseline the compact step is compared
// with.  Cells off the fractal are dead and are written as 0.
//
// Membership of a box cell factorises over levels: the cell is in the
// fractal iff its lowest Lb base-s digits form a member of the level-Lb
// fractal and its digits above Lb form a member of the level-(r-Lb) one.
// Both are precomputed bitmaps (about sqrt of the box each), so a cell's
// membership costs two divisions by s^Lb and two bit look-ups.
//
// Each CTA stages a tile of the box plus a one-cell halo in shared memory,
// one byte per cell (bit 0 = alive member, bit 1 = member), then applies the
// rule from there.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "handle.h"

namespace fr {

static int64_t ipow64(int64_t b, int e)
{
    int64_t v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

// membership of a cell of the level-`levels` fractal (host, digits by hand)
static bool host_member(const fractal *f, int64_t x, int64_t y, int64_t z, int levels)
{
    for (int mu = 0; mu < levels; ++mu) {
        int t = (int)(x % f->s) + f->s * (int)(y % f->s);
        if (f->dim == 3) t += f->s * f->s * (int)(z % f->s);
        x /= f->s; y /= f->s; z /= f->s;
        if (f->dev.hinv[t] < 0) return false;
    }
    return true;
}

static int build_bitmap(const fractal *f, int side, int levels, uint32_t **out, int64_t *words)
{
    int64_t n = ipow64(side, f->dim);
    int64_t nw = (n + 31) / 32;
    std::vector<uint32_t> bits(nw, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t x = i % side, y = (i / side) % side, z = f->dim == 3 ? i / ((int64_t)side * side) : 0;
        if (host_member(f, x, y, z, levels)) bits[i >> 5] |= 1u << (i & 31);
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
    p.S = (int)ipow64(f->s, p.Lb);
    p.C = (int)ipow64(f->s, f->r - p.Lb);
    int rc = build_bitmap(f, p.S, p.Lb, &p.local_bits, &p.local_words);
    if (!rc) rc = build_bitmap(f, p.C, f->r - p.Lb, &p.coarse_bits, &p.coarse_words);
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
                const int64_t li = lx + (int64_t)a.S * (ly + (int64_t)a.S * lz);
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

int launch_bb_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                   uint32_t survive, cudaStream_t st)
{
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
