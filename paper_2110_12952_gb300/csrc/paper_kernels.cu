// paper_kernels.cu -- the paper's own two GPU approaches, kept as baselines
// next to the tiled compact step (Sec. 4, the three approaches compared):
//
//   * "lambda(omega)": the state stays in the n^dim bounding box, but only
//     the blocks of threads the fractal needs are launched: block b is the
//     coarse cell lambda(b) of the fractal at level r - l, a rho^dim group of
//     threads (rho = s^l) covering that cell's rho^dim box cells; threads on
//     members read their Moore neighbours straight from the box.
//   * "nu(omega)" with blocked storage (Sec. 3, the blocked approach and its
//     figure): the state is k^(r-l) mini boxes of rho^dim bytes, one per
//     coarse cell in compact order, each a small bounding box of its level-l
//     sub-fractal.  A block stages its mini box in shared memory and maps the
//     coarse cells of its 3^dim - 1 neighbours once (coarse lambda, a move,
//     coarse nu: the maps are evaluated per block, not per thread); threads
//     on members read neighbours inside the block from shared memory and
//     across the block's edge from the neighbouring mini boxes.
//
// Cells off the fractal hold 0 in both layouts and are written 0.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "handle.h"

namespace fr {

static int pk_fail(const std::string &msg)
{
    set_error(FR_EINVAL, msg);
    return FR_EINVAL;
}

// The local geometry of a blocked layout: rho = s^l, the local membership
// bitmap (rho^dim bits, x fastest) and its local omega -> mini-box offset.
struct PkLocal {
    int l = -1, rho = 0, vol = 0;       // rho^dim
    int64_t kl = 0;                     // k^l members per mini box
    int64_t coarse = 0;                 // k^(r-l) mini boxes
    uint32_t *bits = nullptr;           // device, (vol + 31) / 32 words
    uint16_t *off = nullptr;            // device, kl entries: local omega -> mini-box offset
    int32_t *nb = nullptr;              // device, coarse x 26: neighbouring mini boxes, -1 none
};

static int pk_local(fractal *f, int l, PkLocal &P)
{
    if (l < 1 || l > f->r) return pk_fail("rho_levels must be in [1, r]");
    int64_t rho = 1, vol = 1, kl = 1, coarse = 1;
    for (int i = 0; i < l; ++i) {
        rho *= f->s;
        kl *= f->k;
    }
    for (int i = 0; i < f->dim; ++i) vol *= rho;
    for (int i = 0; i < f->r - l; ++i) coarse *= f->k;
    if (vol > 1024) return pk_fail("rho^dim must be at most 1024 (one thread per cell of a block)");
    if (coarse >= ((int64_t)1 << 31)) return pk_fail("more than 2^31 blocks at this rho");
    P.l = l;
    P.rho = (int)rho;
    P.vol = (int)vol;
    P.kl = kl;
    P.coarse = coarse;
    std::vector<uint32_t> bits((vol + 31) / 32, 0u);
    std::vector<uint16_t> off((size_t)kl);
    for (int64_t w = 0; w < kl; ++w) {
        int64_t x[3] = {0, 0, 0}, sm = 1, t = w;
        for (int mu = 0; mu < l; ++mu) {
            const int d = (int)(t % f->k);
            t /= f->k;
            for (int i = 0; i < f->dim; ++i) x[i] += sm * f->offsets[d * f->dim + i];
            sm *= f->s;
        }
        const int64_t o = x[0] + rho * (x[1] + rho * x[2]);
        off[(size_t)w] = (uint16_t)o;
        bits[(size_t)(o / 32)] |= 1u << (o % 32);
    }
    FR_CUDA(cudaMalloc(&P.bits, bits.size() * sizeof(uint32_t)));
    FR_CUDA(cudaMemcpy(P.bits, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    FR_CUDA(cudaMalloc(&P.off, off.size() * sizeof(uint16_t)));
    FR_CUDA(cudaMemcpy(P.off, off.data(), off.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    return FR_OK;
}

static void pk_free(PkLocal &P)
{
    cudaFree(P.bits);
    cudaFree(P.off);
    cudaFree(P.nb);
    P = PkLocal();
}

__device__ __forceinline__ bool pk_member(const uint32_t *bits, int o) { return (bits[o >> 5] >> (o & 31)) & 1u; }

__device__ __forceinline__ uint32_t pk_rule(uint32_t alive, int count, uint32_t birth, uint32_t survive)
{
    return alive ? (survive >> count) & 1u : (birth >> count) & 1u;
}

// "lambda(omega)": block b covers the box cells of coarse cell lambda(b).
__global__ void lambda_box_kernel(FracDev F, int l, int rho, int64_t coarse, int64_t side,
                                  const uint32_t *__restrict__ bits, const uint8_t *__restrict__ in,
                                  uint8_t *__restrict__ out, uint32_t birth, uint32_t survive)
{
    const int t = threadIdx.x;
    const int tx = t % rho, ty = (t / rho) % rho, tz = F.dim == 3 ? t / (rho * rho) : 0;
    const bool member = pk_member(bits, t);
    for (int64_t b = blockIdx.x; b < coarse; b += gridDim.x) {
        int32_t c[3];
        lambda64(F, (uint64_t)b, F.r - l, c);
        if (!member) continue;
        const int64_t x = (int64_t)c[0] * rho + tx, y = (int64_t)c[1] * rho + ty,
                      z = F.dim == 3 ? (int64_t)c[2] * rho + tz : 0;
        int count = 0;
        for (int dz = (F.dim == 3 ? -1 : 0); dz <= (F.dim == 3 ? 1 : 0); ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int64_t nx = x + dx, ny = y + dy, nz = z + dz;
                    if (nx < 0 || nx >= side || ny < 0 || ny >= side || nz < 0 || nz >= side) continue;
                    count += in[nx + side * (ny + side * nz)] != 0;
                }
        const int64_t idx = x + side * (y + side * z);
        out[idx] = (uint8_t)pk_rule(in[idx] != 0, count, birth, survive);
    }
}

// neighbouring mini boxes of every coarse cell (3^dim - 1 per cell, the
// Moore directions in (dx, dy[, dz]) order, x fastest, centre skipped)
__global__ void pk_nb_kernel(FracDev F, int l, int64_t coarse, int32_t cside, int32_t *__restrict__ nb)
{
    const int nd = F.dim == 3 ? 27 : 9;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < coarse;
         b += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[3];
        lambda64(F, (uint64_t)b, F.r - l, c);
        int slot = 0;
        for (int q = 0; q < nd; ++q) {
            const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = F.dim == 3 ? q / 9 - 1 : 0;
            if (!dx && !dy && !dz) continue;
            const int32_t qx = c[0] + dx, qy = c[1] + dy, qz = c[2] + dz;
            int64_t v = -1;
            if (qx >= 0 && qx < cside && qy >= 0 && qy < cside && (F.dim == 2 || (qz >= 0 && qz < cside)))
                v = nu_levels(F, qx, qy, F.dim == 3 ? qz : 0, F.r - l);
            nb[b * 26 + slot++] = (int32_t)v;
        }
    }
}

// "nu(omega)" on blocked storage.  The maps are evaluated once per block
// (the neighbour table pk_nb_kernel fills at plan time holds the coarse
// nu of each coarse neighbour); the mini box is staged in shared memory.
__global__ void blocked_step_kernel(int dim, int rho, int vol, int64_t coarse, const uint32_t *__restrict__ bits,
                                    const int32_t *__restrict__ nbt, const uint8_t *__restrict__ in,
                                    uint8_t *__restrict__ out, uint32_t birth, uint32_t survive)
{
    extern __shared__ uint8_t mini[];
    __shared__ int32_t nbs[26];
    const int t = threadIdx.x;
    const int tx = t % rho, ty = (t / rho) % rho, tz = dim == 3 ? t / (rho * rho) : 0;
    const bool member = pk_member(bits, t);
    const int nd = dim == 3 ? 26 : 8;
    for (int64_t b = blockIdx.x; b < coarse; b += gridDim.x) {
        __syncthreads();
        mini[t] = in[b * vol + t];
        for (int q = t; q < nd; q += blockDim.x) nbs[q] = nbt[b * 26 + q];   // blocks of 4 or 8 threads too
        __syncthreads();
        if (!member) {
            out[b * vol + t] = 0;
            continue;
        }
        int count = 0;
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    int nx = tx + dx, ny = ty + dy, nz = tz + dz;
                    const int ox = nx < 0 ? -1 : (nx >= rho ? 1 : 0), oy = ny < 0 ? -1 : (ny >= rho ? 1 : 0),
                              oz = nz < 0 ? -1 : (nz >= rho ? 1 : 0);
                    nx -= ox * rho;
                    ny -= oy * rho;
                    nz -= oz * rho;
                    const int o = nx + rho * (ny + rho * nz);
                    if (!ox && !oy && !oz) {
                        count += mini[o] != 0;
                    } else {
                        const int q = (ox + 1) + 3 * (oy + 1) + (dim == 3 ? 9 * (oz + 1) : 0);
                        const int centre = dim == 3 ? 13 : 4;
                        const int32_t nbk = nbs[q < centre ? q : q - 1];
                        if (nbk >= 0) count += in[(int64_t)nbk * vol + o] != 0;
                    }
                }
        out[b * vol + t] = (uint8_t)pk_rule(mini[t] != 0, count, birth, survive);
    }
}

__global__ void blocked_pack_kernel(int64_t cells, int64_t kl, int vol, const uint16_t *__restrict__ off,
                                    const uint8_t *__restrict__ compact, uint8_t *__restrict__ blocked)
{
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < cells;
         w += (int64_t)gridDim.x * blockDim.x)
        blocked[(w / kl) * vol + off[w % kl]] = compact[w] != 0;
}

__global__ void blocked_unpack_kernel(int64_t cells, int64_t kl, int vol, const uint16_t *__restrict__ off,
                                      const uint8_t *__restrict__ blocked, uint8_t *__restrict__ compact)
{
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < cells;
         w += (int64_t)gridDim.x * blockDim.x)
        compact[w] = blocked[(w / kl) * vol + off[w % kl]] != 0;
}

static int pk_grid(int64_t n, int num_sms, int per_sm = 16)
{
    int64_t g = n;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

static int grow(uint8_t **buf, int64_t *have, int64_t bytes, bool zero)
{
    if (*have >= bytes && *buf) return FR_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    FR_CUDA(cudaMalloc(buf, (size_t)bytes));
    if (zero) FR_CUDA(cudaMemset(*buf, 0, (size_t)bytes));
    *have = bytes;
    return FR_OK;
}

}  // namespace fr

using namespace fr;

// per-handle cache of the last blocked geometry and its scratch
struct PkCache {
    PkLocal loc;
    uint8_t *scratch = nullptr;
    int64_t scratch_bytes = 0;
    bool scratch_is_box = false;
};

static PkCache *pk_cache(fractal *f)
{
    if (!f->paper_aux) f->paper_aux = new PkCache();
    return static_cast<PkCache *>(f->paper_aux);
}

void fr::fr_paper_aux_free(fractal *f)
{
    if (!f->paper_aux) return;
    PkCache *c = static_cast<PkCache *>(f->paper_aux);
    pk_free(c->loc);
    cudaFree(c->scratch);
    delete c;
    f->paper_aux = nullptr;
}

static int pk_prepare(fractal *f, int l, bool need_nb, PkLocal **out)
{
    if (l < 1 || l > f->r) return pk_fail("rho_levels must be in [1, r]");
    if (f->mixed) return pk_fail("the paper's approaches: one transition table for every level only");
    PkCache *c = pk_cache(f);
    if (c->loc.l != l) {
        pk_free(c->loc);
        int rc = pk_local(f, l, c->loc);
        if (rc) {
            pk_free(c->loc);
            return rc;
        }
    }
    if (need_nb && !c->loc.nb) {
        FR_CUDA(cudaMalloc(&c->loc.nb, (size_t)c->loc.coarse * 26 * sizeof(int32_t)));
        int64_t cs = 1;
        for (int i = 0; i < f->r - l; ++i) cs *= f->s;
        pk_nb_kernel<<<pk_grid((c->loc.coarse + 255) / 256, f->num_sms), 256>>>(f->dev, l, c->loc.coarse, (int32_t)cs,
                                                                                 c->loc.nb);
        FR_CUDA(cudaGetLastError());
        FR_CUDA(cudaDeviceSynchronize());
    }
    *out = &c->loc;
    return FR_OK;
}

extern "C" int fractal_blocked_info(fractal_t *f, int rho_levels, int64_t *bytes)
{
    clear_error();
    if (!f || !bytes) return pk_fail("fractal_blocked_info: NULL argument");
    PkLocal *P = nullptr;
    int rc = pk_prepare(f, rho_levels, false, &P);
    if (rc) return rc;
    *bytes = P->coarse * P->vol;
    return FR_OK;
}

extern "C" int fractal_blocked_pack(fractal_t *f, int rho_levels, const uint8_t *compact, uint8_t *blocked,
                                    void *stream)
{
    clear_error();
    if (!f || !compact || !blocked) return pk_fail("fractal_blocked_pack: NULL argument");
    PkLocal *P = nullptr;
    int rc = pk_prepare(f, rho_levels, false, &P);
    if (rc) return rc;
    FR_CUDA(cudaMemsetAsync(blocked, 0, (size_t)(P->coarse * P->vol), (cudaStream_t)stream));
    blocked_pack_kernel<<<pk_grid((f->cells + 255) / 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->cells, P->kl, P->vol, P->off, compact, blocked);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_blocked_unpack(fractal_t *f, int rho_levels, const uint8_t *blocked, uint8_t *compact,
                                      void *stream)
{
    clear_error();
    if (!f || !compact || !blocked) return pk_fail("fractal_blocked_unpack: NULL argument");
    PkLocal *P = nullptr;
    int rc = pk_prepare(f, rho_levels, false, &P);
    if (rc) return rc;
    blocked_unpack_kernel<<<pk_grid((f->cells + 255) / 256, f->num_sms), 256, 0, (cudaStream_t)stream>>>(
        f->cells, P->kl, P->vol, P->off, blocked, compact);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_blocked_step(fractal_t *f, int rho_levels, const uint8_t *in, uint8_t *out, int64_t steps,
                                    uint32_t birth, uint32_t survive, void *stream)
{
    clear_error();
    if (!f || !in || !out) return pk_fail("fractal_blocked_step: NULL argument");
    if (steps < 0) return pk_fail("fractal_blocked_step: steps < 0");
    PkLocal *P = nullptr;
    int rc = pk_prepare(f, rho_levels, true, &P);
    if (rc) return rc;
    const int64_t bytes = P->coarse * P->vol;
    const uint8_t *a = in, *b = out;
    if (a < b + bytes && b < a + bytes) return pk_fail("fractal_blocked_step: in and out overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (steps == 0) {
        FR_CUDA(cudaMemcpyAsync(out, in, (size_t)bytes, cudaMemcpyDeviceToDevice, st));
        return FR_OK;
    }
    PkCache *c = pk_cache(f);
    if (steps > 1) {
        rc = grow(&c->scratch, &c->scratch_bytes, bytes, false);
        if (rc) return rc;
        c->scratch_is_box = false;   // blocked generations overwrite it
    }
    const int grid = pk_grid(P->coarse, f->num_sms, 2048 / P->vol > 0 ? 2048 / P->vol : 1);
    const uint8_t *src = in;
    for (int64_t i = 1; i <= steps; ++i) {
        uint8_t *dst = ((steps - i) % 2 == 0) ? out : c->scratch;
        blocked_step_kernel<<<grid, P->vol, P->vol, st>>>(f->dim, P->rho, P->vol, P->coarse, P->bits, P->nb, src,
                                                           dst, birth, survive);
        FR_CUDA(cudaGetLastError());
        src = dst;
    }
    return FR_OK;
}

extern "C" int fractal_lambda_box_step(fractal_t *f, int rho_levels, const uint8_t *in, uint8_t *out,
                                       int64_t steps, uint32_t birth, uint32_t survive, void *stream)
{
    clear_error();
    if (!f || !in || !out) return pk_fail("fractal_lambda_box_step: NULL argument");
    if (steps < 1) return pk_fail("fractal_lambda_box_step: steps < 1");
    if (f->box_cells < 0) {
        set_error(FR_EOVERFLOW, "fractal_lambda_box_step: n^dim overflows");
        return FR_EOVERFLOW;
    }
    const uint8_t *a = in, *b = out;
    if (a < b + f->box_cells && b < a + f->box_cells) return pk_fail("fractal_lambda_box_step: in and out overlap");
    PkLocal *P = nullptr;
    int rc = pk_prepare(f, rho_levels, false, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    PkCache *c = pk_cache(f);
    if (steps > 1) {
        // a box whose cells off the fractal are 0 and are never written
        if (!c->scratch_is_box || c->scratch_bytes < f->box_cells) {
            cudaFree(c->scratch);
            c->scratch = nullptr;
            c->scratch_bytes = 0;
        }
        rc = grow(&c->scratch, &c->scratch_bytes, f->box_cells, true);
        if (rc) return rc;
        c->scratch_is_box = true;
    }
    const int grid = pk_grid(P->coarse, f->num_sms, 2048 / P->vol > 0 ? 2048 / P->vol : 1);
    const uint8_t *src = in;
    for (int64_t i = 1; i <= steps; ++i) {
        uint8_t *dst = ((steps - i) % 2 == 0) ? out : c->scratch;
        lambda_box_kernel<<<grid, P->vol, 0, st>>>(f->dev, P->l, P->rho, P->coarse, f->side, P->bits, src, dst, birth,
                                                   survive);
        FR_CUDA(cudaGetLastError());
        src = dst;
    }
    return FR_OK;
}
