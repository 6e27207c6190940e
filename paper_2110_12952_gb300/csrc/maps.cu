// maps.cu -- the thread maps lambda and nu over arrays (Sec. 3, Sec. 3.1),
// the paper's multi-dimensional compact coordinate (Eqs. 6-8), compact <->
// box views, and the seeded Bernoulli initial state.
//
// All of it is integer work decoded digit by digit on the CUDA cores with
// multiply-high division by the constants s and k.
#include <cuda_runtime.h>
#include <stdint.h>

#include "handle.h"

namespace fr {

static int grid_for(int64_t n, int block, int num_sms)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

__global__ void lambda_kernel(FracDev F, const int64_t *__restrict__ omega, int64_t count,
                              int64_t cells, int32_t *__restrict__ coords)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t w = omega[e];
        int32_t p[3] = {-1, -1, -1};
        if (w >= 0 && w < cells) lambda64(F, (uint64_t)w, F.r, p);
        for (int i = 0; i < F.dim; ++i) coords[e * F.dim + i] = p[i];
    }
}

__device__ __forceinline__ bool in_box(const FracDev &F, int32_t side, const int32_t *c)
{
    for (int i = 0; i < F.dim; ++i)
        if (c[i] < 0 || c[i] >= side) return false;
    return true;
}

__global__ void nu_kernel(FracDev F, int32_t side, const int32_t *__restrict__ coords,
                          int64_t count, int64_t *__restrict__ omega)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[3] = {0, 0, 0};
        for (int i = 0; i < F.dim; ++i) c[i] = coords[e * F.dim + i];
        omega[e] = in_box(F, side, c) ? nu_levels(F, c[0], c[1], c[2], F.r) : -1;
    }
}

// Eqs. 6-8: component (mu mod dim) gains H_mu * k^floor(mu/dim).
__global__ void nu2d_kernel(FracDev F, int32_t side, const int32_t *__restrict__ coords,
                            int64_t count, int64_t *__restrict__ out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[3] = {0, 0, 0};
        for (int i = 0; i < F.dim; ++i) c[i] = coords[e * F.dim + i];
        int64_t acc[3] = {0, 0, 0};
        bool inside = in_box(F, side, c);
        uint32_t x = c[0], y = c[1], z = c[2];
        int64_t w = 1;
        int axis = 0;
        if (F.mix) {
            // per-level tables: level mu's replica ID, weighted by the replica
            // counts of the earlier levels of the same axis
            int64_t wa[3] = {1, 1, 1};
            for (int mu = 0; inside && mu < F.r; ++mu) {
                const MixLevel &M = F.mix[mu];
                const uint32_t qx = divu(F.sdiv, x), qy = divu(F.sdiv, y);
                uint32_t t = (x - qx * F.s) + (uint32_t)F.s * (y - qy * F.s);
                x = qx;
                y = qy;
                if (F.dim == 3) {
                    const uint32_t qz = divu(F.sdiv, z);
                    t += (uint32_t)(F.s * F.s) * (z - qz * F.s);
                    z = qz;
                }
                const int h = M.hinv[t];
                if (h < 0) inside = false;
                const int a = mu % F.dim;
                acc[a] += (int64_t)h * wa[a];
                wa[a] *= M.k;
            }
            for (int i = 0; i < F.dim; ++i) out[e * F.dim + i] = inside ? acc[i] : -1;
            continue;
        }
        for (int mu = 0; inside && mu < F.r; ++mu) {
            uint32_t qx = divu(F.sdiv, x), qy = divu(F.sdiv, y);
            uint32_t t = (x - qx * F.s) + (uint32_t)F.s * (y - qy * F.s);
            x = qx;
            y = qy;
            if (F.dim == 3) {
                uint32_t qz = divu(F.sdiv, z);
                t += (uint32_t)(F.s * F.s) * (z - qz * F.s);
                z = qz;
            }
            int h = F.hinv[t];
            if (h < 0) inside = false;
            acc[axis] += (int64_t)h * w;
            if (++axis == F.dim) {
                axis = 0;
                w *= F.k;
            }
        }
        for (int i = 0; i < F.dim; ++i) out[e * F.dim + i] = inside ? acc[i] : -1;
    }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the omega-th output for a
// seed is mix(seed + (omega + 1) * gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// 16 cells per thread and per iteration, written as one 16-byte store when
// the destination is aligned.
__global__ void init_kernel(uint8_t *__restrict__ state, int64_t cells, uint64_t seed,
                            uint64_t thr)
{
    const int64_t head = (16 - ((uintptr_t)state & 15)) & 15;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t w0 = (c == 0) ? 0 : head + (c - 1) * 16;
        if (w0 >= cells) break;
        int64_t w1 = (c == 0) ? (head < cells ? head : cells) : (w0 + 16 < cells ? w0 + 16 : cells);
        if (c > 0 && w1 - w0 == 16) {
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint64_t x = splitmix64_at(seed, (uint64_t)(w0 + q * 4 + b));
                    word |= (uint32_t)((x >> 11) < thr) << (8 * b);
                }
                v[q] = word;
            }
            *reinterpret_cast<uint4 *>(state + w0) = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
            for (int64_t w = w0; w < w1; ++w)
                state[w] = (splitmix64_at(seed, (uint64_t)w) >> 11) < thr;
        }
    }
}

__global__ void scatter_kernel(FracDev F, int64_t cells, int64_t side,
                               const uint8_t *__restrict__ compact, uint8_t *__restrict__ box)
{
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < cells;
         w += (int64_t)gridDim.x * blockDim.x) {
        int32_t p[3] = {0, 0, 0};
        lambda64(F, (uint64_t)w, F.r, p);
        int64_t idx = p[0] + side * (p[1] + side * (int64_t)p[2]);
        box[idx] = compact[w] != 0;
    }
}

__global__ void gather_kernel(FracDev F, int64_t cells, int64_t side,
                              const uint8_t *__restrict__ box, uint8_t *__restrict__ compact)
{
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < cells;
         w += (int64_t)gridDim.x * blockDim.x) {
        int32_t p[3] = {0, 0, 0};
        lambda64(F, (uint64_t)w, F.r, p);
        int64_t idx = p[0] + side * (p[1] + side * (int64_t)p[2]);
        compact[w] = box[idx] != 0;
    }
}

__global__ void copy_normalise_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                      int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] != 0;
}

int launch_copy_normalise(const uint8_t *in, uint8_t *out, int64_t n, int num_sms, cudaStream_t st)
{
    if (n == 0) return FR_OK;
    copy_normalise_kernel<<<grid_for(n, 256, num_sms), 256, 0, st>>>(in, out, n);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

// Loads the copy kernel's module now, so that a first launch inside a stream
// capture does not have to.
int preload_copy_kernel()
{
    cudaFuncAttributes fa;
    FR_CUDA(cudaFuncGetAttributes(&fa, copy_normalise_kernel));
    return FR_OK;
}

}  // namespace fr

using namespace fr;

static int fail_null(const char *what)
{
    set_error(FR_EINVAL, std::string(what) + ": NULL argument");
    return FR_EINVAL;
}

extern "C" int fractal_lambda(const fractal_t *f, const int64_t *omega, int64_t count,
                              int32_t *coords, void *stream)
{
    if (!f || (count > 0 && (!omega || !coords))) return fail_null("fractal_lambda");
    if (count < 0) return fail_null("fractal_lambda (count < 0)");
    if (count == 0) return FR_OK;
    lambda_kernel<<<grid_for(count, 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->dev, omega, count, f->cells, coords);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_nu(const fractal_t *f, const int32_t *coords, int64_t count,
                          int64_t *omega, void *stream)
{
    if (!f || (count > 0 && (!omega || !coords))) return fail_null("fractal_nu");
    if (count < 0) return fail_null("fractal_nu (count < 0)");
    if (count == 0) return FR_OK;
    nu_kernel<<<grid_for(count, 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->dev, (int32_t)f->side, coords, count, omega);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_nu2d(const fractal_t *f, const int32_t *coords, int64_t count,
                            int64_t *out, void *stream)
{
    if (!f || (count > 0 && (!out || !coords))) return fail_null("fractal_nu2d");
    if (count < 0) return fail_null("fractal_nu2d (count < 0)");
    if (count == 0) return FR_OK;
    nu2d_kernel<<<grid_for(count, 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->dev, (int32_t)f->side, coords, count, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_init_bernoulli(const fractal_t *f, uint8_t *state, uint64_t seed,
                                      double p, void *stream)
{
    if (!f || !state) return fail_null("fractal_init_bernoulli");
    uint64_t thr;
    if (!(p > 0.0)) thr = 0;
    else if (p >= 1.0) thr = 1ull << 53;
    else thr = (uint64_t)(p * 9007199254740992.0);  // floor(p * 2^53), exact scaling
    int64_t chunks = f->cells / 16 + 2;
    init_kernel<<<grid_for(chunks, 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        state, f->cells, seed, thr);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_scatter_to_box(const fractal_t *f, const uint8_t *compact, uint8_t *box,
                                      void *stream)
{
    if (!f || !compact || !box) return fail_null("fractal_scatter_to_box");
    if (f->box_cells < 0) {
        set_error(FR_EOVERFLOW, "fractal_scatter_to_box: n^dim overflows");
        return FR_EOVERFLOW;
    }
    cudaStream_t st = (cudaStream_t)stream;
    FR_CUDA(cudaMemsetAsync(box, 0, (size_t)f->box_cells, st));
    scatter_kernel<<<grid_for(f->cells, 256, f->num_sms), 256, 0, st>>>(
        f->dev, f->cells, f->side, compact, box);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_gather_from_box(const fractal_t *f, const uint8_t *box, uint8_t *compact,
                                       void *stream)
{
    if (!f || !compact || !box) return fail_null("fractal_gather_from_box");
    gather_kernel<<<grid_for(f->cells, 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->dev, f->cells, f->side, box, compact);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}
