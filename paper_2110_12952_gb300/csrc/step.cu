// step.cu -- the compact stencil step (Sec. 3): every compact cell omega
// finds its embedded coordinate with lambda, probes its Moore neighbours and
// maps them back with nu; the life-like rule of the Sec. 4 benchmark is then
// applied.  Results equal the per-cell definition exactly; the work is
// reorganised per subtree ("tile") so that the per-cell cost is O(1):
//
//   * A tile is the k^L cells sharing their digits above level L: a level-L
//     replica, contiguous in omega, filling an s^L-wide box in the embedding.
//     The local lambda (digits below L) is the same for every tile, so it is
//     computed once on the host and kept in shared memory.
//   * The neighbouring level-L replicas of every tile (coarse lambda, a +-1
//     move, coarse nu over the r - L levels above L) depend only on the
//     fractal, so they are computed once per handle into a table, one row of
//     3^dim - 1 compact tile indices per tile.  Membership factorises over
//     levels: a neighbour cell exists iff its coarse tile exists and its local
//     digits form a local member.
//   * Tiles stream through shared memory with bulk asynchronous copies (TMA)
//     in a multi-stage pipeline: the tile bytes (a 16-byte-aligned superset of
//     its omega range) and its table row arrive on one mbarrier while earlier
//     tiles are being computed.  Results are staged in shared memory and
//     written back with bulk stores; the at most 15 unaligned bytes at each
//     end of a tile are written with plain stores.
//   * The tile's cells are scattered into a shared-memory box with a one-cell
//     halo.  Cells of the box that are not local members stay 0 forever; halo
//     cells that are members and touch a member of the tile (list `ring`) are
//     fetched from the neighbouring tiles.
//   * Neighbour counts, 2D "group" mode: one thread owns a level-G subtree
//     (k^G cells, contiguous in omega, filling an s^G x s^G block with
//     s^G = 3 or 4).  It loads the (s^G+2)-wide window rows of its block as
//     32-bit words and adds them byte-wise (a byte holds a count <= 9, so no
//     carries cross bytes): three row adds give vertical sums, two funnel
//     shifts and adds give the 3x3 sums of a whole block row at once.
//     Other cases ("cell" mode, 3D or other s) read the 3^dim - 1 neighbour
//     bytes of each cell from the box.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "handle.h"
#include "tma.cuh"

namespace fr {

constexpr int kMaxGroup = 16;  // cells per group / block positions (s^G <= 4)

struct StepArgs {
    int64_t KL, NT, cells;
    int Px, Py;            // box row pitch and rows per plane (bytes / rows)
    int nring, nbrw, nstage, stage_bytes, tile_bytes;
    int off_bar, off_box, off_tab, off_out, box_bytes;
    int ntab;              // entries of the shared table (cells or groups)
    int KG;                // cells per group (group mode)
    const uint32_t *tab;   // cell mode: box offset per cell; group mode: window base per group
    const uint32_t *ring;
    const int32_t *nbr;
    uint32_t birth, survive;
    int *status;
    int8_t lid_of_q[kMaxGroup];     // group mode: block position -> cell of the group, -1 none
    int16_t rel_of_lid[kMaxGroup];  // group mode: cell of the group -> offset from window base
};

// --------------------------------------------------------------- host plan

static int64_t ipow(int64_t b, int e)
{
    int64_t v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

static int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

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

static int nbr_width(int dim) { return dim == 3 ? 28 : 8; }  // 26 or 8 entries, 16-byte rows
static int nstages() { return 3; }

// Group mode applies to 2D fractals whose block side s^G is 3 or 4.
static int group_levels(const fractal *f)
{
    if (f->dim != 2) return 0;
    if (f->s == 2) return 2;
    if (f->s == 3 || f->s == 4) return 1;
    return 0;
}

struct Geometry {
    int mode;       // 0 = cell, 3 or 4 = group block side
    int G;          // levels per group
    int64_t B, Px, Py, planes;
    int64_t box_bytes, tab_entries;
};

static Geometry plan_geometry(const fractal *f, int L)
{
    Geometry g;
    g.B = ipow(f->s, L);
    g.G = group_levels(f);
    g.mode = (g.G > 0 && L >= g.G && ipow(f->k, g.G) <= kMaxGroup) ? (int)ipow(f->s, g.G) : 0;
    if (!g.mode) g.G = 0;
    if (g.mode) {
        // rows padded so window words never run past a row; pitch/4 odd
        // spreads the rows of neighbouring blocks over the banks
        g.Px = (g.B + 4 + 3) / 4 * 4;
        if ((g.Px / 4) % 2 == 0) g.Px += 4;
        g.Py = g.B + 2;
        g.planes = 1;
        g.tab_entries = ipow(f->k, L - g.G);
    } else {
        g.Px = g.B + 2;
        g.Py = g.B + 2;
        g.planes = (f->dim == 3) ? g.B + 2 : 1;
        g.tab_entries = ipow(f->k, L);
    }
    g.box_bytes = round16(g.Px * g.Py * g.planes + 16);
    return g;
}

struct Layout {
    int64_t stage_bytes, tile_bytes, off_bar, off_box, box_bytes, off_tab, off_out, total;
};

static Layout plan_layout(const fractal *f, int L)
{
    Layout y;
    Geometry g = plan_geometry(f, L);
    int64_t KL = ipow(f->k, L);
    y.tile_bytes = round16(KL + 32);
    y.stage_bytes = 4 * nbr_width(f->dim) + y.tile_bytes;
    int64_t off = (int64_t)nstages() * y.stage_bytes;
    y.off_bar = off;
    off += 8 * nstages();
    off = round16(off);
    y.off_box = off;
    y.box_bytes = g.box_bytes;
    off += y.box_bytes;
    y.off_tab = off;
    off += round16(4 * g.tab_entries);
    y.off_out = off;
    off += y.tile_bytes;
    y.total = off;
    return y;
}

// Deepest tile whose shared-memory layout fits the budget (deeper tiles
// amortise the halo and the table row over more cells).
static int choose_levels(const fractal *f)
{
    if (f->tile_levels_user >= 0) return f->tile_levels_user;
    const int64_t budget = 100 * 1024;
    int best = 0;
    for (int L = 0; L <= f->r; ++L) {
        if (plan_layout(f, L).total > budget) break;
        best = L;
    }
    while (best < f->r && ipow(f->k, f->r - best) >= ((int64_t)1 << 31)) ++best;
    return best;
}

void free_step_plan(StepPlan &p)
{
    cudaFree(p.pos);
    cudaFree(p.ring);
    cudaFree(p.nbr);
    p = StepPlan();
}

// Table row T: compact tile index of each of the 3^dim - 1 neighbouring
// level-L replicas of tile T, found with the coarse lambda and nu.
__global__ void nbr_table_kernel(FracDev F, int64_t NT, int coarse_levels, int32_t coarse_side,
                                 int nbrw, int32_t *__restrict__ table)
{
    const int ndir = (F.dim == 3) ? 27 : 9;
    for (int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; T < NT;
         T += (int64_t)gridDim.x * blockDim.x) {
        int32_t c[3];
        lambda64(F, (uint64_t)T, coarse_levels, c);
        int slot = 0;
        for (int q = 0; q < ndir; ++q) {
            int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (F.dim == 3) ? q / 9 - 1 : 0;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            int32_t qx = c[0] + dx, qy = c[1] + dy, qz = c[2] + dz;
            int64_t t = -1;
            if (qx >= 0 && qx < coarse_side && qy >= 0 && qy < coarse_side &&
                (F.dim == 2 || (qz >= 0 && qz < coarse_side)))
                t = nu_levels(F, qx, qy, F.dim == 3 ? qz : 0, coarse_levels);
            table[T * nbrw + slot++] = (int32_t)t;
        }
        for (; slot < nbrw; ++slot) table[T * nbrw + slot] = -1;
    }
}

template <int DIM, int SG>
__global__ void step_tma_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in,
                                uint8_t *__restrict__ out);

template <int DIM, int SG>
static int configure(StepPlan &p, int num_sms)
{
    int per_sm = 0;
    FR_CUDA(cudaFuncSetAttribute(step_tma_kernel<DIM, SG>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem));
    FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tma_kernel<DIM, SG>, p.block, p.smem));
    if (per_sm < 1) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    p.grid = (int)std::min<int64_t>((int64_t)per_sm * num_sms, p.NT);
    return FR_OK;
}

int ensure_step_plan(fractal *f)
{
    int L = choose_levels(f);
    if (f->plan.L == L && f->plan.pos) return FR_OK;
    free_step_plan(f->plan);
    int rc = ensure_status(f);
    if (rc) return rc;
    StepPlan p;
    p.L = L;
    p.KL = ipow(f->k, L);
    p.NT = ipow(f->k, f->r - L);
    p.B = (int)ipow(f->s, L);
    p.coarse_levels = f->r - L;
    if (p.NT >= ((int64_t)1 << 31)) {
        set_error(FR_EOVERFLOW, "fractal_step: more than 2^31 tiles at this tile depth");
        return FR_EOVERFLOW;
    }
    const Geometry geo = plan_geometry(f, L);
    const Layout y = plan_layout(f, L);
    p.mode = geo.mode;
    p.G = geo.G;
    p.Px = (int)geo.Px;
    p.Py = (int)geo.Py;
    p.P = p.Px;
    p.box_bytes = (int)y.box_bytes;
    p.stage_bytes = (int)y.stage_bytes;
    p.tile_bytes = (int)y.tile_bytes;
    p.off_bar = (int)y.off_bar;
    p.off_box = (int)y.off_box;
    p.off_pos = (int)y.off_tab;
    p.off_out = (int)y.off_out;
    p.smem = (int)y.total;
    p.nstage = nstages();
    p.nbrw = nbr_width(f->dim);
    p.ntab = (int)geo.tab_entries;
    const int dim = f->dim;
    const int64_t W[3] = {geo.B + 2, geo.B + 2, dim == 3 ? geo.B + 2 : 1};  // padded extents
    auto offset_of = [&](const int b[3]) -> int64_t {
        return b[0] + geo.Px * (b[1] + geo.Py * (int64_t)(dim == 3 ? b[2] : 0));
    };
    if (geo.Px * geo.Py * geo.planes >= (1 << 24)) {
        set_error(FR_EINVAL, "fractal_step: tile box too large");
        return FR_EINVAL;
    }

    // local lambda -> padded box offset; occupancy of the interior
    std::vector<uint32_t> pos(p.KL);
    std::vector<uint8_t> occ((size_t)(geo.Px * geo.Py * geo.planes), 0);
    for (int64_t l = 0; l < p.KL; ++l) {
        int c[3];
        host_lambda(f, l, L, c);
        int b[3] = {c[0] + 1, c[1] + 1, c[2] + 1};
        int64_t o = offset_of(b);
        pos[l] = (uint32_t)o;
        occ[o] = 1;
    }
    std::vector<uint32_t> tab;
    if (p.mode) {
        // group g = cells [g k^G, (g+1) k^G); its block sits at s^G * (coarse
        // lambda of g over L - G levels); the window starts one cell up-left
        const int KG = (int)ipow(f->k, p.G), SG = p.mode;
        p.KG = KG;
        for (int q = 0; q < kMaxGroup; ++q) p.lid_of_q[q] = -1;
        for (int lid = 0; lid < KG; ++lid) {
            int c[3];
            host_lambda(f, lid, p.G, c);
            p.lid_of_q[c[1] * SG + c[0]] = (int8_t)lid;
            p.rel_of_lid[lid] = (int16_t)((c[1] + 1) * geo.Px + (c[0] + 1));
        }
        tab.resize(geo.tab_entries);
        for (int64_t g = 0; g < geo.tab_entries; ++g) {
            int c[3];
            host_lambda(f, g, L - p.G, c);
            tab[g] = (uint32_t)((int64_t)c[1] * SG * geo.Px + (int64_t)c[0] * SG);
        }
    } else {
        tab = pos;
    }
    // halo ring: padded cells with some coordinate 0 or B+1 that are members
    // of their (wrapped) local box and touch an interior member
    std::vector<uint32_t> ring;
    const int centre = (dim == 3) ? 13 : 4;
    for (int64_t bz = 0; bz < W[2]; ++bz)
        for (int64_t by = 0; by < W[1]; ++by)
            for (int64_t bx = 0; bx < W[0]; ++bx) {
                int b[3] = {(int)bx, (int)by, (int)bz};
                bool halo = false;
                int dir = 0, m3 = 1, q[3] = {0, 0, 0};
                for (int i = 0; i < dim; ++i) {
                    int d = (b[i] == 0) ? -1 : (b[i] == W[i] - 1 ? 1 : 0);
                    if (d) halo = true;
                    dir += (d + 1) * m3;
                    m3 *= 3;
                    q[i] = (b[i] == 0) ? p.B - 1 : (b[i] == W[i] - 1 ? 0 : b[i] - 1);
                }
                if (!halo) continue;
                int64_t lw = host_nu(f, q, L);
                if (lw < 0) continue;
                bool touches = false;
                const int nq = (dim == 3) ? 27 : 9;
                for (int e = 0; e < nq && !touches; ++e) {
                    int dd[3] = {e % 3 - 1, (e / 3) % 3 - 1, e / 9 - 1};
                    int nb[3] = {0, 0, 0};
                    bool inside = true;
                    for (int i = 0; i < dim; ++i) {
                        nb[i] = b[i] + dd[i];
                        if (nb[i] < 1 || nb[i] > W[i] - 2) inside = false;
                    }
                    if (inside && occ[offset_of(nb)]) touches = true;
                }
                if (!touches) continue;
                const int slot = dir < centre ? dir : dir - 1;
                ring.push_back((uint32_t)offset_of(b) | ((uint32_t)slot << 24));
                ring.push_back((uint32_t)lw);
            }
    p.nring = (int)(ring.size() / 2);
    FR_CUDA(cudaMalloc(&p.pos, tab.size() * sizeof(uint32_t)));
    FR_CUDA(cudaMemcpy(p.pos, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    if (!ring.empty()) {
        FR_CUDA(cudaMalloc(&p.ring, ring.size() * sizeof(uint32_t)));
        FR_CUDA(cudaMemcpy(p.ring, ring.data(), ring.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    // neighbour-tile table
    cudaError_t e = cudaMalloc(&p.nbr, (size_t)p.NT * p.nbrw * sizeof(int32_t));
    if (e != cudaSuccess) {
        free_step_plan(p);
        return cuda_fail(e, "fractal_step: neighbour table allocation");
    }
    {
        int64_t g = std::min<int64_t>((p.NT + 255) / 256, (int64_t)f->num_sms * 16);
        nbr_table_kernel<<<(int)std::max<int64_t>(g, 1), 256>>>(
            f->dev, p.NT, p.coarse_levels, (int32_t)ipow(f->s, p.coarse_levels), p.nbrw, p.nbr);
        FR_CUDA(cudaGetLastError());
        FR_CUDA(cudaDeviceSynchronize());
    }
    p.block = 256;
    if (dim == 3) rc = configure<3, 0>(p, f->num_sms);
    else if (p.mode == 4) rc = configure<2, 4>(p, f->num_sms);
    else if (p.mode == 3) rc = configure<2, 3>(p, f->num_sms);
    else rc = configure<2, 0>(p, f->num_sms);
    if (rc) {
        free_step_plan(p);
        return rc;
    }
    f->plan = p;
    return FR_OK;
}

// ------------------------------------------------------------------ kernel

// Issue the bulk loads of tile T into one stage: the table row and the
// 16-byte-aligned part of the tile's bytes that lies inside the buffer.
__device__ __forceinline__ void issue_tile(const StepArgs &a, const uint8_t *in, int64_t T,
                                           uint8_t *stage, uint64_t *bar)
{
    const uintptr_t start = (uintptr_t)(in + T * a.KL);
    const uintptr_t end = start + (uintptr_t)a.KL;
    const uintptr_t lo = start & ~(uintptr_t)15;
    const uintptr_t in_lo = ((uintptr_t)in + 15) & ~(uintptr_t)15;
    const uintptr_t in_hi = ((uintptr_t)in + (uintptr_t)a.cells) & ~(uintptr_t)15;
    uintptr_t b0 = lo > in_lo ? lo : in_lo;
    uintptr_t b1 = ((end + 15) & ~(uintptr_t)15);
    if (b1 > in_hi) b1 = in_hi;
    const uint32_t row_bytes = 4u * (uint32_t)a.nbrw;
    const uint32_t data_bytes = b1 > b0 ? (uint32_t)(b1 - b0) : 0u;
    mbar_arrive_expect_tx(bar, row_bytes + data_bytes);
    bulk_g2s(stage, a.nbr + T * a.nbrw, row_bytes, bar);
    if (data_bytes) bulk_g2s(stage + row_bytes + (b0 - lo), (const void *)b0, data_bytes, bar);
}

__device__ __forceinline__ uint32_t lds32(const uint8_t *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

// Group mode: new states of the k^G cells of one group from its window.
template <int SG>
__device__ __forceinline__ void group_compute(const StepArgs &a, const uint8_t *box, uint32_t base,
                                              uint8_t *gout)
{
    constexpr int R = SG + 2;
    uint32_t lo[R], hi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t ad = base + r * a.Px;
        const uint32_t al = ad & ~3u;
        const uint32_t w0 = lds32(box + al), w1 = lds32(box + al + 4);
        const uint32_t sh = (ad & 3u) * 8u;
        lo[r] = __funnelshift_r(w0, w1, sh);
        hi[r] = w1 >> sh;
    }
#pragma unroll
    for (int j = 0; j < SG; ++j) {
        const uint32_t vl = lo[j] + lo[j + 1] + lo[j + 2];
        const uint32_t vh = hi[j] + hi[j + 1] + hi[j + 2];
        // byte c: 3x3 sum (centre included) around block column c
        const uint32_t sum = vl + __funnelshift_r(vl, vh, 8) + __funnelshift_r(vl, vh, 16);
        const uint32_t alive = __funnelshift_r(lo[j + 1], hi[j + 1], 8);
#pragma unroll
        for (int c = 0; c < SG; ++c) {
            const int lid = a.lid_of_q[j * SG + c];
            if (lid >= 0) {
                const uint32_t al = (alive >> (8 * c)) & 1u;
                const uint32_t cnt = ((sum >> (8 * c)) & 0xffu) - al;
                gout[lid] = ((al ? a.survive : a.birth) >> cnt) & 1u;
            }
        }
    }
}

template <int DIM, int SG>
__global__ void __launch_bounds__(256)
step_tma_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + a.off_bar);
    uint8_t *box = smem + a.off_box;
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + a.off_tab);
    uint8_t *ostage = smem + a.off_out;
    constexpr int NDIR = (DIM == 3) ? 27 : 9;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t G = gridDim.x;
    const uint32_t row_bytes = 4u * (uint32_t)a.nbrw;

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
        fence_proxy_async_smem();
        for (int s = 0; s < a.nstage; ++s) {
            int64_t T = blockIdx.x + s * G;
            if (T < a.NT) issue_tile(a, in, T, smem + s * a.stage_bytes, &bars[s]);
        }
    }
    for (int i = tid; i < a.box_bytes / 16; i += nth)
        reinterpret_cast<uint4 *>(box)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < a.ntab; i += nth) tab[i] = a.tab[i];
    __syncthreads();

    int nb[NDIR - 1];
    if (SG == 0) {
        const int PX = a.Px, PXY = a.Px * a.Py;
        int e = 0;
        for (int q = 0; q < NDIR; ++q) {
            int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (DIM == 3) ? q / 9 - 1 : 0;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            nb[e++] = dx + PX * dy + PXY * dz;
        }
    }

    const uintptr_t in_lo = ((uintptr_t)in + 15) & ~(uintptr_t)15;
    const uintptr_t in_hi = ((uintptr_t)in + (uintptr_t)a.cells) & ~(uintptr_t)15;

    int64_t i = 0;
    for (int64_t T = blockIdx.x; T < a.NT; T += G, ++i) {
        const int s = (int)(i % a.nstage);
        const uint32_t parity = (uint32_t)((i / a.nstage) & 1);
        uint8_t *stage = smem + s * a.stage_bytes;
        const int32_t *nrow = reinterpret_cast<const int32_t *>(stage);
        const bool ok = mbar_wait_bounded(&bars[s], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.status, FR_ETIMEOUT);
            break;
        }
        const uintptr_t start = (uintptr_t)(in + T * a.KL);
        const uintptr_t end = start + (uintptr_t)a.KL;
        const uintptr_t lo = start & ~(uintptr_t)15;
        uint8_t *data = stage + row_bytes;           // data[j] <-> address lo + j
        // bytes of the tile the bulk copy could not cover (unaligned buffer ends)
        uintptr_t b0 = lo > in_lo ? lo : in_lo;
        uintptr_t b1 = (end + 15) & ~(uintptr_t)15;
        if (b1 > in_hi) b1 = in_hi;
        if (b0 > start || b1 < end) {
            for (int64_t l = tid; l < a.KL; l += nth) {
                uintptr_t ad = start + l;
                if (ad < b0 || ad >= b1) data[ad - lo] = *(const uint8_t *)ad;
            }
            __syncthreads();
        }
        const uint8_t *tin = data + (start - lo);
        if (SG == 0) {
            for (int64_t l = tid; l < a.KL; l += nth) box[tab[l]] = tin[l] != 0;
        } else {
            for (int g = tid; g < a.ntab; g += nth) {
                const uint32_t base = tab[g];
                const uint8_t *src = tin + (int64_t)g * a.KG;
                for (int lid = 0; lid < a.KG; ++lid) box[base + a.rel_of_lid[lid]] = src[lid] != 0;
            }
        }
        for (int e = tid; e < a.nring; e += nth) {
            const uint32_t w0 = __ldg(a.ring + 2 * e), lw = __ldg(a.ring + 2 * e + 1);
            const int32_t t = nrow[w0 >> 24];
            uint8_t v = 0;
            if (t >= 0) v = in[(int64_t)t * a.KL + lw] != 0;
            box[w0 & 0xffffff] = v;
        }
        if (tid == 0) bulk_wait_read_all();   // previous tile's bulk store has read ostage
        __syncthreads();
        // stage s is consumed: refill it with the tile nstage iterations ahead
        if (tid == 0) {
            const int64_t Tn = T + a.nstage * G;
            fence_proxy_async_smem();
            if (Tn < a.NT) issue_tile(a, in, Tn, stage, &bars[s]);
        }
        const uintptr_t ostart = (uintptr_t)(out + T * a.KL);
        const uintptr_t oend = ostart + (uintptr_t)a.KL;
        const uintptr_t olo = ostart & ~(uintptr_t)15;
        uint8_t *tout = ostage + (ostart - olo);
        if (SG == 0) {
            for (int64_t l = tid; l < a.KL; l += nth) {
                const int p = tab[l];
                int cnt = 0;
#pragma unroll
                for (int e = 0; e < NDIR - 1; ++e) cnt += box[p + nb[e]];
                const uint32_t mask = box[p] ? a.survive : a.birth;
                tout[l] = (mask >> cnt) & 1u;
            }
        } else {
            for (int g = tid; g < a.ntab; g += nth)
                group_compute<(SG > 0 ? SG : 3)>(a, box, tab[g], tout + (int64_t)g * a.KG);
        }
        __syncthreads();
        const uintptr_t c0 = (ostart + 15) & ~(uintptr_t)15;
        const uintptr_t c1 = oend & ~(uintptr_t)15;
        if (tid == 0) {
            fence_proxy_async_smem();
            if (c1 > c0) {
                bulk_s2g((void *)c0, ostage + (c0 - olo), (uint32_t)(c1 - c0));
                bulk_commit();
            }
        }
        // unaligned head and tail bytes
        if (c1 > c0) {
            const int head = (int)(c0 - ostart), tail = (int)(oend - c1);
            if (tid < head) *(uint8_t *)(ostart + tid) = tout[tid];
            else if (tid >= 32 && tid < 32 + tail) {
                const int j = tid - 32;
                *(uint8_t *)(c1 + j) = ostage[c1 - olo + j];
            }
        } else {
            for (int64_t l = tid; l < a.KL; l += nth) *(uint8_t *)(ostart + l) = tout[l];
        }
    }
    if (tid == 0) bulk_wait_all();
}

int launch_step_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                     uint32_t survive, cudaStream_t st)
{
    const StepPlan &p = f->plan;
    StepArgs a;
    a.KL = p.KL;
    a.NT = p.NT;
    a.cells = f->cells;
    a.Px = p.Px;
    a.Py = p.Py;
    a.nring = p.nring;
    a.nbrw = p.nbrw;
    a.nstage = p.nstage;
    a.stage_bytes = p.stage_bytes;
    a.tile_bytes = p.tile_bytes;
    a.off_bar = p.off_bar;
    a.off_box = p.off_box;
    a.off_tab = p.off_pos;
    a.off_out = p.off_out;
    a.box_bytes = p.box_bytes;
    a.ntab = p.ntab;
    a.KG = p.KG;
    a.tab = p.pos;
    a.ring = p.ring;
    a.nbr = p.nbr;
    a.birth = birth;
    a.survive = survive;
    a.status = f->status;
    for (int q = 0; q < kMaxGroup; ++q) {
        a.lid_of_q[q] = p.lid_of_q[q];
        a.rel_of_lid[q] = p.rel_of_lid[q];
    }
    if (f->dim == 3)
        step_tma_kernel<3, 0><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == 4)
        step_tma_kernel<2, 4><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == 3)
        step_tma_kernel<2, 3><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else
        step_tma_kernel<2, 0><<<p.grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

}  // namespace fr
