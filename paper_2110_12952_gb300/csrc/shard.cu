// shard.cu -- one instance split over several shards (one per GPU): shard g
// owns a contiguous range of the instance's tiles (level-L subtrees, k^L
// cells each, in omega order; whole replicas of the levels above when the
// split falls on their boundaries, Sec. 3) and each generation receives,
// from the shards that own them, the neighbouring tiles that its tiles'
// Moore neighbourhoods reach (its halo).  The plan is computed on the host
// from the coarse lambda and nu of the tiles (no GPU needed); the device part
// gathers the tiles a peer needs into a send buffer and runs the step over
// the shard's own tiles with a neighbour table that points into its halo.
// Moving the send buffers between shards (NCCL send/recv, or a peer copy) is
// the caller's: it is plain data movement.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "handle.h"

struct fractal_shard {
    int k = 0, s = 0, r = 0, dim = 0, L = 0;
    std::vector<int32_t> offsets;
    int nshards = 0, shard = 0;
    int64_t KL = 0, NT = 0;             // cells per tile, tiles of the instance
    int ndir = 0, nbrw = 0;             // neighbour directions, table row width
    std::vector<int64_t> bounds;        // nshards + 1 tile boundaries
    int64_t t0 = 0, nlocal = 0, nhalo = 0;
    std::vector<int32_t> table;         // nlocal x nbrw, slots of this shard's buffer, -1 none
    std::vector<std::vector<int64_t>> send;   // per peer: global tiles it needs from this shard
    std::vector<int64_t> send_dst;      // per peer: first cell of their block in the peer's buffer
    std::vector<std::vector<int64_t>> recv;   // per peer: global tiles received from it
    std::vector<int64_t> recv_dst;      // per peer: first cell of their block in this buffer
    // device side (fractal_shard_attach)
    fractal *f = nullptr;
    int32_t *d_table = nullptr;
    std::vector<int32_t *> d_send;      // per peer: local tile indices to gather
};

namespace fr {

static int shard_fail(int code, const std::string &msg)
{
    set_error(code, msg);
    return code;
}

// coarse lambda of tile T over `levels` levels (the tile's box position in
// units of s^L)
static void tile_lambda(const fractal_shard *p, int64_t T, int levels, int64_t c[3])
{
    c[0] = c[1] = c[2] = 0;
    int64_t sm = 1;
    for (int mu = 0; mu < levels; ++mu) {
        const int d = (int)(T % p->k);
        T /= p->k;
        for (int i = 0; i < p->dim; ++i) c[i] += sm * p->offsets[d * p->dim + i];
        sm *= p->s;
    }
}

// coarse nu: the tile at box position c, or -1 (outside the box or off the
// fractal); `hinv` maps a digit tuple to its replica
static int64_t tile_nu(const fractal_shard *p, const std::vector<int> &hinv, const int64_t q[3], int levels)
{
    int64_t side = 1;
    for (int mu = 0; mu < levels; ++mu) side *= p->s;
    int64_t x[3] = {q[0], q[1], q[2]};
    for (int i = 0; i < p->dim; ++i)
        if (x[i] < 0 || x[i] >= side) return -1;
    int64_t w = 0, km = 1;
    for (int mu = 0; mu < levels; ++mu) {
        int t = 0, m = 1;
        for (int i = 0; i < p->dim; ++i) {
            t += (int)(x[i] % p->s) * m;
            x[i] /= p->s;
            m *= p->s;
        }
        const int h = hinv[t];
        if (h < 0) return -1;
        w += h * km;
        km *= p->k;
    }
    return w;
}

static int owner_of(const fractal_shard *p, int64_t T)
{
    return (int)(std::upper_bound(p->bounds.begin(), p->bounds.end(), T) - p->bounds.begin()) - 1;
}

__global__ void shard_pack_kernel(const uint8_t *__restrict__ buf, const int32_t *__restrict__ tiles,
                                  int64_t ntiles, int64_t KL, uint8_t *__restrict__ send)
{
    // one tile per block iteration; consecutive threads copy consecutive bytes
    for (int64_t j = blockIdx.x; j < ntiles; j += gridDim.x) {
        const uint8_t *src = buf + (int64_t)tiles[j] * KL;
        uint8_t *dst = send + j * KL;
        for (int64_t b = threadIdx.x; b < KL; b += blockDim.x) dst[b] = src[b];
    }
}

}  // namespace fr

using namespace fr;

extern "C" int fractal_shard_plan(int k, int s, int r, int dim, const int32_t *offsets, int tile_levels,
                                  int nshards, int shard, fractal_shard_t **out)
{
    clear_error();
    if (!out || !offsets) return shard_fail(FR_EINVAL, "fractal_shard_plan: NULL argument");
    *out = nullptr;
    if (dim != 2 && dim != 3) return shard_fail(FR_EINVAL, "fractal_shard_plan: dim must be 2 or 3");
    if (s < 2 || s > 16 || k < 1 || r < 0)
        return shard_fail(FR_EINVAL, "fractal_shard_plan: bad k, s or r");
    int sd = 1;
    for (int i = 0; i < dim; ++i) sd *= s;
    if (k > sd) return shard_fail(FR_EINVAL, "fractal_shard_plan: k > s^dim");
    if (tile_levels < 0 || tile_levels > r)
        return shard_fail(FR_EINVAL, "fractal_shard_plan: tile_levels must be in [0, r]");
    if (nshards < 1 || shard < 0 || shard >= nshards)
        return shard_fail(FR_EINVAL, "fractal_shard_plan: need 0 <= shard < nshards");
    std::vector<int> hinv(sd, -1);
    for (int j = 0; j < k; ++j) {
        int t = 0, m = 1;
        for (int i = 0; i < dim; ++i) {
            const int v = offsets[j * dim + i];
            if (v < 0 || v >= s) return shard_fail(FR_EINVAL, "fractal_shard_plan: offset outside [0,s)");
            t += v * m;
            m *= s;
        }
        if (hinv[t] >= 0) return shard_fail(FR_EINVAL, "fractal_shard_plan: duplicate offset rows");
        hinv[t] = j;
    }
    fractal_shard *p = new (std::nothrow) fractal_shard();
    if (!p) return shard_fail(FR_ENOMEM, "fractal_shard_plan: out of host memory");
    p->k = k; p->s = s; p->r = r; p->dim = dim; p->L = tile_levels;
    p->offsets.assign(offsets, offsets + (size_t)k * dim);
    p->nshards = nshards;
    p->shard = shard;
    p->KL = 1;
    for (int i = 0; i < tile_levels; ++i) p->KL *= k;
    p->NT = 1;
    const int C = r - tile_levels;
    for (int i = 0; i < C; ++i) p->NT *= k;
    p->ndir = dim == 3 ? 26 : 8;
    p->nbrw = dim == 3 ? 28 : 8;
    if (p->NT < nshards) {
        delete p;
        return shard_fail(FR_EINVAL, "fractal_shard_plan: fewer tiles than shards (lower tile_levels)");
    }
    if (p->NT * p->ndir > ((int64_t)1 << 28) || p->NT >= ((int64_t)1 << 31)) {
        delete p;
        return shard_fail(FR_EOVERFLOW, "fractal_shard_plan: too many tiles (raise tile_levels)");
    }
    // contiguous, equal tile ranges
    p->bounds.resize(nshards + 1);
    for (int g = 0; g <= nshards; ++g) p->bounds[g] = p->NT * g / nshards;
    p->t0 = p->bounds[shard];
    p->nlocal = p->bounds[shard + 1] - p->t0;

    // the instance's neighbour-tile table (coarse lambda, a Moore move, coarse nu)
    std::vector<int32_t> nb((size_t)(p->NT * p->ndir));
    for (int64_t T = 0; T < p->NT; ++T) {
        int64_t c[3];
        tile_lambda(p, T, C, c);
        int slot = 0;
        for (int q = 0; q < (dim == 3 ? 27 : 9); ++q) {
            const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = dim == 3 ? q / 9 - 1 : 0;
            if (!dx && !dy && !dz) continue;
            const int64_t n[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
            nb[(size_t)(T * p->ndir + slot++)] = (int32_t)tile_nu(p, hinv, n, C);
        }
    }
    // for every shard pair (g, h): how many tiles of g touch h; then the
    // halo block of g inside h's buffer follows h's own tiles, ordered by g
    std::vector<int64_t> cnt((size_t)nshards * nshards, 0);
    std::vector<int> seen;
    for (int64_t T = 0; T < p->NT; ++T) {
        const int g = owner_of(p, T);
        seen.clear();
        for (int d = 0; d < p->ndir; ++d) {
            const int32_t tn = nb[(size_t)(T * p->ndir + d)];
            if (tn < 0) continue;
            const int h = owner_of(p, tn);
            if (h != g && std::find(seen.begin(), seen.end(), h) == seen.end()) seen.push_back(h);
        }
        for (int h : seen) ++cnt[(size_t)g * nshards + h];
    }
    auto block_start = [&](int g, int h) {   // first halo slot of g's tiles in h's buffer
        int64_t slot = p->bounds[h + 1] - p->bounds[h];
        for (int g2 = 0; g2 < g; ++g2)
            if (g2 != h) slot += cnt[(size_t)g2 * nshards + h];
        return slot;
    };
    p->send.assign(nshards, {});
    p->recv.assign(nshards, {});
    p->send_dst.assign(nshards, 0);
    p->recv_dst.assign(nshards, 0);
    // this shard's sends (ascending tiles) and halo (ascending per owner)
    for (int64_t T = p->t0; T < p->t0 + p->nlocal; ++T) {
        seen.clear();
        for (int d = 0; d < p->ndir; ++d) {
            const int32_t tn = nb[(size_t)(T * p->ndir + d)];
            if (tn < 0) continue;
            const int h = owner_of(p, tn);
            if (h == shard) continue;
            if (std::find(seen.begin(), seen.end(), h) == seen.end()) {
                seen.push_back(h);
                p->send[h].push_back(T);
            }
            p->recv[h].push_back(tn);
        }
    }
    std::unordered_map<int64_t, int32_t> slot_of;
    p->nhalo = 0;
    for (int g = 0; g < nshards; ++g) {
        auto &v = p->recv[g];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        if (g == shard) continue;
        p->send_dst[g] = block_start(shard, g) * p->KL;
        p->recv_dst[g] = block_start(g, shard) * p->KL;
        if ((int64_t)v.size() != cnt[(size_t)g * nshards + shard] ||
            (int64_t)p->send[g].size() != cnt[(size_t)shard * nshards + g]) {
            delete p;
            return shard_fail(FR_EINVAL, "fractal_shard_plan: tile adjacency is not symmetric");
        }
        const int64_t base = block_start(g, shard);
        for (size_t i = 0; i < v.size(); ++i) slot_of[v[i]] = (int32_t)(base + (int64_t)i);
        p->nhalo += (int64_t)v.size();
    }
    p->table.assign((size_t)(p->nlocal * p->nbrw), -1);
    for (int64_t i = 0; i < p->nlocal; ++i)
        for (int d = 0; d < p->ndir; ++d) {
            const int32_t tn = nb[(size_t)((p->t0 + i) * p->ndir + d)];
            int32_t v = -1;
            if (tn >= 0) v = owner_of(p, tn) == shard ? (int32_t)(tn - p->t0) : slot_of.at(tn);
            p->table[(size_t)(i * p->nbrw + d)] = v;
        }
    *out = p;
    return FR_OK;
}

extern "C" int fractal_shard_destroy(fractal_shard_t *p)
{
    clear_error();
    if (!p) return FR_OK;
    if (p->d_table || !p->d_send.empty()) cudaDeviceSynchronize();
    cudaFree(p->d_table);
    for (int32_t *d : p->d_send) cudaFree(d);
    delete p;
    return FR_OK;
}

extern "C" int fractal_shard_info(const fractal_shard_t *p, int64_t *first_cell, int64_t *local_cells,
                                  int64_t *buffer_cells)
{
    clear_error();
    if (!p) return shard_fail(FR_EINVAL, "fractal_shard_info: NULL plan");
    if (first_cell) *first_cell = p->t0 * p->KL;
    if (local_cells) *local_cells = p->nlocal * p->KL;
    if (buffer_cells) *buffer_cells = (p->nlocal + p->nhalo) * p->KL;
    return FR_OK;
}

static int list_out(const std::vector<int64_t> &v, int64_t *tiles, int64_t capacity, int64_t *count)
{
    if (count) *count = (int64_t)v.size();
    if (tiles) {
        if (capacity < (int64_t)v.size()) return shard_fail(FR_EINVAL, "fractal_shard: capacity too small");
        std::copy(v.begin(), v.end(), tiles);
    }
    return FR_OK;
}

extern "C" int fractal_shard_sends(const fractal_shard_t *p, int peer, int64_t *tiles, int64_t capacity,
                                   int64_t *count, int64_t *dst_cell)
{
    clear_error();
    if (!p || peer < 0 || peer >= p->nshards) return shard_fail(FR_EINVAL, "fractal_shard_sends: bad argument");
    if (dst_cell) *dst_cell = p->send_dst[peer];
    return list_out(p->send[peer], tiles, capacity, count);
}

extern "C" int fractal_shard_recvs(const fractal_shard_t *p, int peer, int64_t *tiles, int64_t capacity,
                                   int64_t *count, int64_t *dst_cell)
{
    clear_error();
    if (!p || peer < 0 || peer >= p->nshards) return shard_fail(FR_EINVAL, "fractal_shard_recvs: bad argument");
    if (dst_cell) *dst_cell = p->recv_dst[peer];
    return list_out(p->recv[peer], tiles, capacity, count);
}

extern "C" int fractal_shard_neighbours(const fractal_shard_t *p, int32_t *table, int64_t capacity)
{
    clear_error();
    if (!p || !table) return shard_fail(FR_EINVAL, "fractal_shard_neighbours: NULL argument");
    const int64_t n = p->nlocal * p->ndir;
    if (capacity < n) return shard_fail(FR_EINVAL, "fractal_shard_neighbours: capacity too small");
    for (int64_t i = 0; i < p->nlocal; ++i)
        for (int d = 0; d < p->ndir; ++d) table[i * p->ndir + d] = p->table[(size_t)(i * p->nbrw + d)];
    return FR_OK;
}

extern "C" int fractal_shard_attach(fractal_shard_t *p, fractal_t *f)
{
    clear_error();
    if (!p || !f) return shard_fail(FR_EINVAL, "fractal_shard_attach: NULL argument");
    if (f->mixed || f->k != p->k || f->s != p->s || f->r != p->r || f->dim != p->dim || f->offsets != p->offsets)
        return shard_fail(FR_EINVAL, "fractal_shard_attach: the handle is not the plan's fractal");
    if (f->server_refs.load() > 0)
        return shard_fail(FR_EBUSY, "fractal_shard_attach: a server still holds requests on this handle");
    if (f->tile_levels_user != p->L) {
        f->tile_levels_user = p->L;
        cudaDeviceSynchronize();
        free_step_plan(f->plan);
    }
    int rc = ensure_step_plan(f);
    if (rc) return rc;
    cudaFree(p->d_table);
    p->d_table = nullptr;
    for (int32_t *d : p->d_send) cudaFree(d);
    p->d_send.assign(p->nshards, nullptr);
    FR_CUDA(cudaMalloc(&p->d_table, std::max<size_t>(1, p->table.size()) * sizeof(int32_t)));
    FR_CUDA(cudaMemcpy(p->d_table, p->table.data(), p->table.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    for (int g = 0; g < p->nshards; ++g) {
        if (p->send[g].empty()) continue;
        std::vector<int32_t> local(p->send[g].size());
        for (size_t i = 0; i < local.size(); ++i) local[i] = (int32_t)(p->send[g][i] - p->t0);
        FR_CUDA(cudaMalloc(&p->d_send[g], local.size() * sizeof(int32_t)));
        FR_CUDA(cudaMemcpy(p->d_send[g], local.data(), local.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    p->f = f;
    return FR_OK;
}

extern "C" int fractal_shard_pack(const fractal_shard_t *p, int peer, const uint8_t *buffer, uint8_t *send,
                                  void *stream)
{
    clear_error();
    if (!p || !buffer || peer < 0 || peer >= p->nshards)
        return shard_fail(FR_EINVAL, "fractal_shard_pack: bad argument");
    if (!p->f) return shard_fail(FR_EINVAL, "fractal_shard_pack: plan not attached to a handle");
    const int64_t n = (int64_t)p->send[peer].size();
    if (n == 0) return FR_OK;
    if (!send) return shard_fail(FR_EINVAL, "fractal_shard_pack: NULL send buffer");
    const int grid = (int)std::min<int64_t>(n, (int64_t)p->f->num_sms * 8);
    shard_pack_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(buffer, p->d_send[peer], n, p->KL, send);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_shard_step(fractal_shard_t *p, const uint8_t *in, uint8_t *out, uint32_t birth,
                                  uint32_t survive, void *stream)
{
    clear_error();
    if (!p || !in || !out) return shard_fail(FR_EINVAL, "fractal_shard_step: NULL argument");
    if (!p->f) return shard_fail(FR_EINVAL, "fractal_shard_step: plan not attached to a handle");
    const int64_t cells = (p->nlocal + p->nhalo) * p->KL;
    const uint8_t *a = in, *b = out;
    if (a < b + cells && b < a + cells) return shard_fail(FR_EINVAL, "fractal_shard_step: in and out overlap");
    fractal *f = p->f;
    if (f->plan.L != p->L) return shard_fail(FR_EINVAL, "fractal_shard_step: the handle was re-planned");
    return launch_step_tiles(f, in, out, p->d_table, p->nlocal, cells, birth, survive, (cudaStream_t)stream);
}
