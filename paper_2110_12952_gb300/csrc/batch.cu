// batch.cu -- batched execution of many independent, uneven instances
// (fractal_batch_*): the pending generations of all instances are fused into
// one launch per class and generation, and the whole run is captured into a
// single CUDA graph that is replayed with one launch.  The arithmetic is the
// per-instance step of step.cu, unchanged.
//
// A class is a set of instances whose fractals share the per-tile tables:
// the same transition table (k, s, dim, offsets) and the same tile depth L.
// Each class launch walks the concatenation of its instances' tiles; the
// instance of every tile comes from a tile -> instance map.  Instances are
// ordered by decreasing step count, so the instances still running at
// generation j are a prefix of the class list and each launch covers that
// prefix.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "handle.h"
#include "step.h"

extern "C" const char *fractal_last_error(void);

namespace fr {

struct BatchInst {
    fractal *f;
    const uint8_t *in;
    uint8_t *out;
    int64_t steps;
    uint32_t birth, survive;
};

struct BatchClass {
    fractal *rep;                   // a handle whose plan serves the class
    std::vector<int> members;       // instance indices, steps descending
    std::vector<int64_t> active_tiles;  // [j] = tiles of the instances with steps >= j (j >= 1)
    std::vector<int> active_count;      // [j] = number of those instances
    size_t desc_off = 0, map_off = 0;   // offsets in the device arena
};

}  // namespace fr

struct fractal_batch {
    std::vector<fr::BatchInst> insts;
    std::vector<fr::BatchClass> classes;
    uint8_t *arena = nullptr;       // descriptors, tile maps, ping-pong scratch
    size_t arena_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;     // private capture stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool dirty = true;
    int64_t last_updates = 0;
    int last_launches = 0;
};

namespace fr {

static int bfail(int code, const std::string &m)
{
    set_error(code, m);
    return code;
}

static void drop_graph(fractal_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Key of the per-tile tables of a planned handle.
static std::string class_key(const fractal *f)
{
    std::string k = std::to_string(f->k) + "," + std::to_string(f->s) + "," +
                    std::to_string(f->dim) + "," + std::to_string(f->plan.L) + "," +
                    std::to_string(f->plan.mode) + "|";
    for (int32_t v : f->offsets) k += std::to_string(v) + ",";
    for (int32_t v : f->lev_k) k += "l" + std::to_string(v);   // per-level tables
    return k;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Build classes, descriptors and tile maps, and capture the graph.
static int build(fractal_batch *b)
{
    drop_graph(b);
    b->classes.clear();
    int rc;
    for (auto &in : b->insts) {
        rc = ensure_step_plan(in.f);
        if (rc) return rc;
    }
    std::map<std::string, int> cls_of;
    for (int i = 0; i < (int)b->insts.size(); ++i) {
        const BatchInst &in = b->insts[i];
        if (in.steps <= 0) continue;
        const std::string key = class_key(in.f);
        auto it = cls_of.find(key);
        if (it == cls_of.end()) {
            it = cls_of.emplace(key, (int)b->classes.size()).first;
            BatchClass c;
            c.rep = in.f;
            b->classes.push_back(c);
        }
        b->classes[it->second].members.push_back(i);
    }
    // arena layout: per class descriptors and tile map, then per instance scratch
    size_t off = 0;
    int64_t max_steps = 0;
    for (auto &c : b->classes) {
        std::stable_sort(c.members.begin(), c.members.end(),
                         [&](int x, int y) { return b->insts[x].steps > b->insts[y].steps; });
        int64_t tiles = 0;
        for (int i : c.members) tiles += b->insts[i].f->plan.NT;
        if (tiles >= ((int64_t)1 << 31)) return bfail(FR_EOVERFLOW, "fractal_batch_run: too many tiles in one class");
        c.desc_off = off;
        off = al256(off + c.members.size() * sizeof(InstDesc));
        c.map_off = off;
        off = al256(off + (size_t)tiles * sizeof(int32_t));
        max_steps = std::max(max_steps, b->insts[c.members.front()].steps);
    }
    std::vector<size_t> scratch_off(b->insts.size(), 0);
    for (size_t i = 0; i < b->insts.size(); ++i) {
        if (b->insts[i].steps <= 1) continue;
        scratch_off[i] = off;
        off = al256(off + (size_t)b->insts[i].f->cells);
    }
    if (off > b->arena_bytes) {
        cudaFree(b->arena);
        b->arena = nullptr;
        b->arena_bytes = 0;
        cudaError_t e = cudaMalloc(&b->arena, off ? off : 256);
        if (e != cudaSuccess) return cuda_fail(e, "fractal_batch_run: arena allocation");
        b->arena_bytes = off;
    }
    // descriptors and maps
    for (auto &c : b->classes) {
        std::vector<InstDesc> d(c.members.size());
        std::vector<int32_t> map;
        int64_t t0 = 0;
        for (size_t q = 0; q < c.members.size(); ++q) {
            const BatchInst &in = b->insts[c.members[q]];
            uint8_t *scratch = b->arena + scratch_off[c.members[q]];
            // generation j writes `out` when steps - j is even, so the last
            // generation lands in `out`; generation 1 reads `in`
            uint8_t *odd = (in.steps % 2 == 1) ? in.out : scratch;
            uint8_t *even = (in.steps % 2 == 1) ? scratch : in.out;
            d[q].first = in.in;
            d[q].odd_dst = odd;
            d[q].even_dst = even;
            d[q].nbr = in.f->plan.nbr;
            d[q].cells = in.f->cells;
            d[q].tile0 = t0;
            make_rule(in.birth, in.survive, &d[q].rule);
            map.insert(map.end(), (size_t)in.f->plan.NT, (int32_t)q);
            t0 += in.f->plan.NT;
        }
        c.active_tiles.assign(max_steps + 1, 0);
        c.active_count.assign(max_steps + 1, 0);
        for (size_t q = 0; q < c.members.size(); ++q) {
            const BatchInst &in = b->insts[c.members[q]];
            for (int64_t j = 1; j <= in.steps; ++j) {
                c.active_count[j] = (int)q + 1;
                c.active_tiles[j] = d[q].tile0 + in.f->plan.NT;
            }
        }
        cudaError_t e = cudaMemcpy(b->arena + c.desc_off, d.data(), d.size() * sizeof(InstDesc),
                                   cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->arena + c.map_off, map.data(), map.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "fractal_batch_run: table upload");
    }
    // capture: generation by generation, one launch per class
    if (!b->cap) {
        FR_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        FR_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
        FR_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    }
    rc = preload_copy_kernel();
    if (rc) return rc;
    cudaGraph_t graph = nullptr;
    FR_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    int64_t updates = 0;
    int lrc = FR_OK;
    std::string where;
    for (size_t i = 0; i < b->insts.size() && !lrc; ++i)
        if (b->insts[i].steps == 0) {
            lrc = launch_copy_normalise(b->insts[i].in, b->insts[i].out, b->insts[i].f->cells,
                                        b->insts[i].f->num_sms, b->cap);
            if (lrc) where = "copy of instance " + std::to_string(i);
            ++launches;
        }
    for (int64_t j = 1; j <= max_steps && !lrc; ++j)
        for (size_t ci = 0; ci < b->classes.size() && !lrc; ++ci) {
            const BatchClass &c = b->classes[ci];
            const int m = c.active_count[j];
            if (m == 0) continue;
            lrc = launch_step_multi(c.rep, reinterpret_cast<const InstDesc *>(b->arena + c.desc_off),
                                    reinterpret_cast<const int32_t *>(b->arena + c.map_off), m,
                                    c.active_tiles[j], (int)j, b->cap);
            if (lrc)
                where = "class " + std::to_string(ci) + " (L=" + std::to_string(c.rep->plan.L) +
                        ", mode " + std::to_string(c.rep->plan.mode) + ") generation " + std::to_string(j);
            ++launches;
        }
    if (lrc) {
        const std::string msg = fractal_last_error();
        set_error(lrc, "fractal_batch_run: launch failed at " + where + " (launch " +
                           std::to_string(launches) + "): " + msg);
    }
    for (auto &in : b->insts) updates += in.f->cells * in.steps;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (lrc) {
        if (graph) cudaGraphDestroy(graph);
        return lrc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "fractal_batch_run: stream capture");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "fractal_batch_run: graph instantiation");
    b->last_launches = launches;
    b->last_updates = updates;
    b->dirty = false;
    return FR_OK;
}

}  // namespace fr

using namespace fr;

extern "C" int fractal_batch_create(fractal_batch_t **out)
{
    if (!out) return bfail(FR_EINVAL, "fractal_batch_create: out is NULL");
    *out = new (std::nothrow) fractal_batch();
    if (!*out) return bfail(FR_ENOMEM, "fractal_batch_create: out of host memory");
    return FR_OK;
}

extern "C" int fractal_batch_destroy(fractal_batch_t *b)
{
    if (!b) return FR_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    cudaFree(b->arena);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
    return FR_OK;
}

extern "C" int fractal_batch_add(fractal_batch_t *b, fractal_t *f, const uint8_t *in, uint8_t *out,
                                 int64_t steps, uint32_t birth, uint32_t survive, int64_t *id)
{
    if (!b || !f || !in || !out) return bfail(FR_EINVAL, "fractal_batch_add: NULL argument");
    if (steps < 0) return bfail(FR_EINVAL, "fractal_batch_add: steps < 0");
    const uint8_t *o = out;
    if (in < o + f->cells && o < in + f->cells)
        return bfail(FR_EINVAL, "fractal_batch_add: in and out overlap");
    BatchInst bi{f, in, out, steps, birth, survive};
    b->insts.push_back(bi);
    b->dirty = true;
    if (id) *id = (int64_t)b->insts.size() - 1;
    return FR_OK;
}

extern "C" int fractal_batch_clear(fractal_batch_t *b)
{
    if (!b) return bfail(FR_EINVAL, "fractal_batch_clear: NULL argument");
    cudaDeviceSynchronize();
    drop_graph(b);
    b->insts.clear();
    b->classes.clear();
    b->dirty = true;
    return FR_OK;
}

extern "C" int fractal_batch_run(fractal_batch_t *b, void *stream)
{
    if (!b) return bfail(FR_EINVAL, "fractal_batch_run: NULL argument");
    if (b->insts.empty()) return FR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->dirty) {
        int rc = build(b);
        if (rc) return rc;
    }
    FR_CUDA(cudaGraphLaunch(b->exec, st));
    return FR_OK;
}

extern "C" int fractal_batch_stats(const fractal_batch_t *b, int64_t *updates, int64_t *launches)
{
    if (!b) return bfail(FR_EINVAL, "fractal_batch_stats: NULL argument");
    if (updates) *updates = b->last_updates;
    if (launches) *launches = b->last_launches;
    return FR_OK;
}
