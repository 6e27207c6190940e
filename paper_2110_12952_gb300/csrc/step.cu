// step.cu -- the compact stencil step (Sec. 3): every compact cell omega
// finds its embedded coordinate with lambda, probes its Moore neighbours and
// maps them back with nu; the life-like rule of the Sec. 4 benchmark is then
// applied.  Results equal the per-cell definition exactly; the work is
// reorganised per subtree ("tile") so that the per-cell cost is O(1):
//
//   * A tile is the k^L cells sharing their digits above level L: a level-L
//     replica, contiguous in omega, filling an s^L-wide box in the embedding.
//     The local lambda (digits below L) is the same for every tile, so it is
//     computed once on the host into `pos` and kept in shared memory.
//   * The tile's cells are scattered into a shared-memory box with a one-cell
//     halo.  Cells of the box that are not local members stay 0 forever.
//   * The halo comes from the 3^dim - 1 neighbouring level-L replicas.  Their
//     compact tile indices are found once per tile with the coarse lambda/nu
//     over the r - L levels above L (membership factorises over levels, so a
//     neighbour cell exists iff its coarse tile exists and its local digits
//     are a local member).  Only halo cells that are members and touch a
//     member of the tile are fetched (list `ring`, built on the host).
//   * Each cell then reads its 3^dim - 1 neighbours from the box and writes
//     its new state back in omega order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "handle.h"

namespace fr {

struct StepArgs {
    int64_t KL, NT;
    int P, box_bytes, coarse_levels, nring;
    int32_t coarse_side;   // s^(r-L)
    const uint32_t *pos;
    const uint32_t *ring;
    uint32_t birth, survive;
};

// --------------------------------------------------------------- host plan

static int64_t ipow(int64_t b, int e)
{
    int64_t v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

// local lambda over L levels on the host
static void host_lambda(const fractal *f, int64_t l, int L, int p[3])
{
    p[0] = p[1] = p[2] = 0;
    int64_t sm = 1;
    for (int mu = 0; mu < L; ++mu) {
        int d = (int)(l % f->k);
        l /= f->k;
        for (int i = 0; i < f->dim; ++i) p[i] += (int)(sm * f->offsets[d * f->dim + i]);
        sm *= f->s;
    }
}

// local nu over L levels on the host (-1 if not a local member)
static int64_t host_nu(const fractal *f, const int q[3], int L)
{
    int x[3] = {q[0], q[1], q[2]};
    int64_t w = 0, km = 1;
    for (int mu = 0; mu < L; ++mu) {
        int t = 0, m = 1;
        for (int i = 0; i < f->dim; ++i) {
            t += (x[i] % f->s) * m;
            x[i] /= f->s;
            m *= f->s;
        }
        int h = f->dev.hinv[t];
        if (h < 0) return -1;
        w += h * km;
        km *= f->k;
    }
    return w;
}

static int plan_smem(const fractal *f, int L, int64_t *box_bytes_out)
{
    int64_t B = ipow(f->s, L), P = B + 2;
    int64_t box = ipow(P, f->dim);
    box = (box + 15) / 16 * 16;
    int64_t KL = ipow(f->k, L);
    *box_bytes_out = box;
    int64_t total = box + 4 * KL;
    return total > (1 << 30) ? (1 << 30) : (int)total;
}

static int choose_levels(const fractal *f)
{
    if (f->tile_levels_user >= 0) return f->tile_levels_user;
    const int budget = 64 * 1024;
    int best = 0;
    for (int L = 0; L <= f->r; ++L) {
        int64_t bb;
        if (plan_smem(f, L, &bb) <= budget && ipow(f->k, L) <= (1 << 20)) best = L;
        else break;
    }
    return best;
}

void free_step_plan(StepPlan &p)
{
    cudaFree(p.pos);
    cudaFree(p.ring);
    p = StepPlan();
}

template <int DIM>
__global__ void step_tiled_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in,
                                  uint8_t *__restrict__ out);

int ensure_step_plan(fractal *f)
{
    int L = choose_levels(f);
    if (f->plan.L == L && f->plan.pos) return FR_OK;
    free_step_plan(f->plan);
    StepPlan p;
    p.L = L;
    p.KL = ipow(f->k, L);
    p.NT = ipow(f->k, f->r - L);
    p.B = (int)ipow(f->s, L);
    p.P = p.B + 2;
    int64_t box_bytes;
    p.smem = plan_smem(f, L, &box_bytes);
    p.box_bytes = (int)box_bytes;
    p.coarse_levels = f->r - L;
    const int dim = f->dim;
    const int P = p.P;
    int64_t boxn = ipow(P, dim);

    // local lambda -> padded box offset; occupancy of the interior
    std::vector<uint32_t> pos(p.KL);
    std::vector<uint8_t> occ(boxn, 0);
    for (int64_t l = 0; l < p.KL; ++l) {
        int c[3];
        host_lambda(f, l, L, c);
        int64_t o = (c[0] + 1) + (int64_t)P * ((c[1] + 1) + (dim == 3 ? (int64_t)P * (c[2] + 1) : 0));
        pos[l] = (uint32_t)o;
        occ[o] = 1;
    }
    // halo ring: box cells with some coordinate 0 or P-1
    std::vector<uint32_t> ring;
    int q[3] = {0, 0, 0};
    for (int64_t o = 0; o < boxn; ++o) {
        int64_t t = o;
        int b[3] = {0, 0, 0};
        for (int i = 0; i < dim; ++i) {
            b[i] = (int)(t % P);
            t /= P;
        }
        bool halo = false;
        int dir = 0, m3 = 1;
        for (int i = 0; i < dim; ++i) {
            int d = (b[i] == 0) ? -1 : (b[i] == P - 1 ? 1 : 0);
            if (d) halo = true;
            dir += (d + 1) * m3;
            m3 *= 3;
            q[i] = (b[i] == 0) ? p.B - 1 : (b[i] == P - 1 ? 0 : b[i] - 1);
        }
        if (!halo) continue;
        int64_t lw = host_nu(f, q, L);
        if (lw < 0) continue;
        // touches an interior member?
        bool touches = false;
        int nq = (dim == 3) ? 27 : 9;
        for (int e = 0; e < nq && !touches; ++e) {
            int dd[3] = {e % 3 - 1, (e / 3) % 3 - 1, e / 9 - 1};
            int nb[3];
            bool inside = true;
            for (int i = 0; i < dim; ++i) {
                nb[i] = b[i] + dd[i];
                if (nb[i] < 1 || nb[i] > P - 2) inside = false;
            }
            if (!inside) continue;
            int64_t no = nb[0] + (int64_t)P * (nb[1] + (dim == 3 ? (int64_t)P * nb[2] : 0));
            if (occ[no]) touches = true;
        }
        if (!touches) continue;
        ring.push_back((uint32_t)o | ((uint32_t)dir << 24));
        ring.push_back((uint32_t)lw);
    }
    if (boxn >= (1 << 24)) {
        set_error(FR_EINVAL, "fractal_step: tile box too large");
        return FR_EINVAL;
    }
    p.nring = (int)(ring.size() / 2);
    FR_CUDA(cudaMalloc(&p.pos, pos.size() * sizeof(uint32_t)));
    FR_CUDA(cudaMemcpy(p.pos, pos.data(), pos.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    if (!ring.empty()) {
        FR_CUDA(cudaMalloc(&p.ring, ring.size() * sizeof(uint32_t)));
        FR_CUDA(cudaMemcpy(p.ring, ring.data(), ring.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    // launch shape: persistent CTAs, as many as fit
    p.block = 256;
    int per_sm = 1;
    if (dim == 2) {
        FR_CUDA(cudaFuncSetAttribute(step_tiled_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem));
        FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tiled_kernel<2>, p.block, p.smem));
    } else {
        FR_CUDA(cudaFuncSetAttribute(step_tiled_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem));
        FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tiled_kernel<3>, p.block, p.smem));
    }
    if (per_sm < 1) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    int64_t g = (int64_t)per_sm * f->num_sms;
    p.grid = (int)std::min<int64_t>(g, p.NT);
    f->plan = p;
    return FR_OK;
}

// ------------------------------------------------------------------ kernel

template <int DIM>
__global__ void __launch_bounds__(256)
step_tiled_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *box = smem;
    uint32_t *pos = reinterpret_cast<uint32_t *>(smem + a.box_bytes);
    __shared__ long long ntile[27];
    constexpr int NDIR = (DIM == 3) ? 27 : 9;
    const int tid = threadIdx.x, nth = blockDim.x;

    for (int i = tid; i < a.box_bytes / 16; i += nth)
        reinterpret_cast<uint4 *>(box)[i] = make_uint4(0, 0, 0, 0);
    for (int64_t l = tid; l < a.KL; l += nth) pos[l] = a.pos[l];
    __syncthreads();

    const int P = a.P;
    const int PP = P * P;
    int nb[26];
    {
        int e = 0;
        for (int q = 0; q < NDIR; ++q) {
            int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (DIM == 3) ? q / 9 - 1 : 0;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            nb[e++] = dx + P * dy + PP * dz;
        }
    }

    for (int64_t T = blockIdx.x; T < a.NT; T += gridDim.x) {
        // neighbour tiles through the coarse maps over levels L..r-1
        if (tid < NDIR) {
            int32_t c[3];
            lambda64(F, (uint64_t)T, a.coarse_levels, c);
            int dx = tid % 3 - 1, dy = (tid / 3) % 3 - 1, dz = (DIM == 3) ? tid / 9 - 1 : 0;
            int32_t qx = c[0] + dx, qy = c[1] + dy, qz = c[2] + dz;
            long long t = -1;
            if (qx >= 0 && qx < a.coarse_side && qy >= 0 && qy < a.coarse_side &&
                (DIM == 2 || (qz >= 0 && qz < a.coarse_side)))
                t = nu_levels(F, qx, qy, DIM == 3 ? qz : 0, a.coarse_levels);
            ntile[tid] = t;
        }
        const uint8_t *tin = in + T * a.KL;
        for (int64_t l = tid; l < a.KL; l += nth) box[pos[l]] = tin[l] != 0;
        __syncthreads();
        for (int e = tid; e < a.nring; e += nth) {
            uint32_t w0 = a.ring[2 * e], lw = a.ring[2 * e + 1];
            long long t = ntile[w0 >> 24];
            uint8_t v = 0;
            if (t >= 0) v = in[t * a.KL + lw] != 0;
            box[w0 & 0xffffff] = v;
        }
        __syncthreads();
        uint8_t *tout = out + T * a.KL;
        for (int64_t l = tid; l < a.KL; l += nth) {
            const int p = pos[l];
            int cnt = 0;
#pragma unroll
            for (int e = 0; e < NDIR - 1; ++e) cnt += box[p + nb[e]];
            const uint32_t mask = box[p] ? a.survive : a.birth;
            tout[l] = (mask >> cnt) & 1u;
        }
        __syncthreads();
    }
}

int launch_step_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                     uint32_t survive, cudaStream_t st)
{
    const StepPlan &p = f->plan;
    StepArgs a;
    a.KL = p.KL;
    a.NT = p.NT;
    a.P = p.P;
    a.box_bytes = p.box_bytes;
    a.coarse_levels = p.coarse_levels;
    a.nring = p.nring;
    a.coarse_side = (int32_t)ipow(f->s, p.coarse_levels);
    a.pos = p.pos;
    a.ring = p.ring;
    a.birth = birth;
    a.survive = survive;
    if (f->dim == 2)
        step_tiled_kernel<2><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else
        step_tiled_kernel<3><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

}  // namespace fr
