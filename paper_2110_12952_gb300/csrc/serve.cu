// serve.cu -- continuous-batching request server (fractal_server_*).
//
// Requests (a fractal handle, a seed and density for the initial state, a
// number of generations, a rule) arrive at any time.  A worker thread owns
// the device side:
//   * admission: queued requests become resident, in arrival order, while
//     their two state buffers (2 k^r bytes) fit in the server's HBM budget;
//     buffers come from the stream-ordered allocator on the server stream;
//   * ticks: every resident request advances by min(chunk, remaining)
//     generations; one tick is one launch per class (same fractal tables and
//     tile depth) and generation, with the multi-instance step of step.cu, so
//     requests that arrived while others run share the same launches;
//   * retirement: a finished request's final state is copied to its host
//     buffer (or reduced to its live-cell count), its buffers are released on
//     the stream, and its completion is stamped when the copy has landed.
// The arithmetic is the per-instance step, unchanged: a served result equals
// fractal_step on the same initial state.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.h"
#include "step.h"

extern "C" int fractal_init_bernoulli(const fractal_t *f, uint8_t *state_dev, uint64_t seed,
                                      double p, void *stream);
extern "C" const char *fractal_last_error(void);

namespace fr {

static double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { kQueued = 0, kResident = 1, kRetiring = 2, kDone = 3, kFailed = 4 };

struct Request {
    int64_t id;
    fractal *f;
    uint64_t seed;
    double p;
    int64_t steps, remaining;
    uint32_t birth, survive;
    uint8_t *host_out;
    uint8_t *buf[2] = {nullptr, nullptr};
    int cur = 0;                 // buffer holding the state
    int64_t bytes = 0;           // device bytes held
    int64_t population = -1;     // live cells of the result (when no host buffer)
    int64_t *pop_host = nullptr; // pinned slot receiving the population
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = kQueued;
};

__global__ void population_kernel(const uint8_t *__restrict__ s, int64_t n,
                                  unsigned long long *__restrict__ out)
{
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += s[i] != 0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

struct UploadSlot {
    uint8_t *dev = nullptr, *host = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool used = false;
};

}  // namespace fr

struct fractal_server {
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread worker;
    bool stop = false;
    std::deque<fr::Request *> queue;
    std::vector<fr::Request *> resident, retiring;
    std::unordered_map<int64_t, fr::Request *> all;
    int64_t next_id = 0;
    int64_t budget = 0, used = 0;
    int chunk = 8;
    int device = 0;
    cudaStream_t st = nullptr;
    fr::UploadSlot slots[3];
    int64_t tick = 0;
    int64_t *pop_ring = nullptr;   // pinned live-cell counts
    int64_t pop_cap = 1 << 16;
    // statistics
    int64_t admitted = 0, completed = 0, ticks = 0, launches = 0, updates = 0;
    double gpu_first = -1, gpu_last = 0;
    int error = FR_OK;
    std::string error_msg;
};

namespace fr {

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

static std::string class_key(const fractal *f)
{
    std::string k = std::to_string(f->k) + "," + std::to_string(f->s) + "," +
                    std::to_string(f->dim) + "," + std::to_string(f->plan.L) + "," +
                    std::to_string(f->plan.mode) + "|";
    for (int32_t v : f->offsets) k += std::to_string(v) + ",";
    for (int32_t v : f->lev_k) k += "l" + std::to_string(v);   // per-level tables
    return k;
}

static int fail_srv(fractal_server *s, int code, const std::string &m)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->error) {
            s->error = code;
            s->error_msg = m;
        }
    }
    s->done_cv.notify_all();
    return code;
}

// Runs on the CUDA runtime's callback thread when the stream reaches the end
// of a request's result copy: stamps the completion and releases its budget.
struct Landing {
    fractal_server *s;
    Request *r;
};

static void CUDART_CB on_landed(void *arg)
{
    Landing *L = static_cast<Landing *>(arg);
    fractal_server *s = L->s;
    Request *r = L->r;
    const double td = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->t_done = td;
        if (!r->host_out) r->population = *r->pop_host;
        r->state = kDone;
        r->f->server_refs.fetch_sub(1);
        s->used -= r->bytes;
        ++s->completed;
        s->gpu_last = td;
        s->retiring.erase(std::remove(s->retiring.begin(), s->retiring.end(), r), s->retiring.end());
    }
    delete L;
    s->done_cv.notify_all();
    s->cv.notify_one();
}

// One tick: advance every resident request by min(chunk, remaining).
static int run_tick(fractal_server *s, std::vector<Request *> &res)
{
    struct Cls {
        fractal *rep;
        std::vector<Request *> m;
    };
    std::map<std::string, Cls> classes;
    for (Request *r : res) {
        auto &c = classes[class_key(r->f)];
        c.rep = r->f;
        c.m.push_back(r);
    }
    // per class: requests by decreasing generations this tick
    size_t need = 0;
    for (auto &kv : classes) {
        auto &m = kv.second.m;
        std::stable_sort(m.begin(), m.end(), [&](Request *a, Request *b) {
            return std::min<int64_t>(a->remaining, s->chunk) > std::min<int64_t>(b->remaining, s->chunk);
        });
        int64_t tiles = 0;
        for (Request *r : m) tiles += r->f->plan.NT;
        need = al256(need + m.size() * sizeof(InstDesc));
        need = al256(need + (size_t)tiles * sizeof(int32_t));
    }
    UploadSlot &u = s->slots[s->tick % 3];
    if (u.used) {
        cudaError_t e = cudaEventSynchronize(u.ev);   // the tick that used this slot has finished
        if (e != cudaSuccess) return cuda_fail(e, "fractal_server: tick wait");
    }
    if (need > u.cap) {
        cudaFree(u.dev);
        cudaFreeHost(u.host);
        u.dev = nullptr;
        u.host = nullptr;
        size_t cap = std::max(need * 2, (size_t)1 << 20);
        cudaError_t e = cudaMalloc(&u.dev, cap);
        if (e == cudaSuccess) e = cudaMallocHost(&u.host, cap);
        if (e != cudaSuccess) return cuda_fail(e, "fractal_server: upload buffers");
        u.cap = cap;
    }
    struct Launch {
        fractal *rep;
        size_t desc_off, map_off;
        std::vector<int> count;
        std::vector<int64_t> tiles;
    };
    std::vector<Launch> ls;
    size_t off = 0;
    int gmax = 0;
    for (auto &kv : classes) {
        auto &m = kv.second.m;
        Launch L;
        L.rep = kv.second.rep;
        L.desc_off = off;
        InstDesc *d = reinterpret_cast<InstDesc *>(u.host + off);
        off = al256(off + m.size() * sizeof(InstDesc));
        L.map_off = off;
        int32_t *map = reinterpret_cast<int32_t *>(u.host + off);
        int64_t t0 = 0;
        const int c0 = (int)std::min<int64_t>(m.front()->remaining, s->chunk);
        L.count.assign(c0 + 1, 0);
        L.tiles.assign(c0 + 1, 0);
        for (size_t q = 0; q < m.size(); ++q) {
            Request *r = m[q];
            const int c = (int)std::min<int64_t>(r->remaining, s->chunk);
            d[q].first = r->buf[r->cur];
            d[q].odd_dst = r->buf[1 - r->cur];
            d[q].even_dst = r->buf[r->cur];
            d[q].nbr = r->f->plan.nbr;
            d[q].cells = r->f->cells;
            d[q].tile0 = t0;
            make_rule(r->birth, r->survive, &d[q].rule);
            std::fill(map + t0, map + t0 + r->f->plan.NT, (int32_t)q);
            t0 += r->f->plan.NT;
            for (int j = 1; j <= c; ++j) {
                L.count[j] = (int)q + 1;
                L.tiles[j] = t0;
            }
        }
        off = al256(off + (size_t)t0 * sizeof(int32_t));
        gmax = std::max(gmax, c0);
        ls.push_back(std::move(L));
    }
    FR_CUDA(cudaMemcpyAsync(u.dev, u.host, off, cudaMemcpyHostToDevice, s->st));
    for (int j = 1; j <= gmax; ++j)
        for (auto &L : ls) {
            if (j >= (int)L.count.size() || L.count[j] == 0) continue;
            int rc = launch_step_multi(L.rep, reinterpret_cast<const InstDesc *>(u.dev + L.desc_off),
                                       reinterpret_cast<const int32_t *>(u.dev + L.map_off), L.count[j],
                                       L.tiles[j], j, s->st);
            if (rc) return rc;
            ++s->launches;
        }
    FR_CUDA(cudaEventRecord(u.ev, s->st));
    u.used = true;
    ++s->tick;
    ++s->ticks;
    for (Request *r : res) {
        const int64_t c = std::min<int64_t>(r->remaining, s->chunk);
        if (c % 2 == 1) r->cur = 1 - r->cur;
        r->remaining -= c;
        s->updates += c * r->f->cells;
    }
    return FR_OK;
}

static int retire(fractal_server *s, Request *r)
{
    if (r->host_out) {
        FR_CUDA(cudaMemcpyAsync(r->host_out, r->buf[r->cur], (size_t)r->f->cells,
                                cudaMemcpyDeviceToHost, s->st));
    } else {
        // live-cell count, reduced into the spare buffer's first bytes
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(r->buf[1 - r->cur]);
        FR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s->st));
        const int64_t n = r->f->cells;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)r->f->num_sms * 8));
        population_kernel<<<grid, 256, 0, s->st>>>(r->buf[r->cur], n, cnt);
        FR_CUDA(cudaGetLastError());
        r->pop_host = s->pop_ring + (r->id % s->pop_cap);
        FR_CUDA(cudaMemcpyAsync(r->pop_host, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
    }
    FR_CUDA(cudaFreeAsync(r->buf[0], s->st));
    r->buf[0] = r->buf[1] = nullptr;
    r->state = kRetiring;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->retiring.push_back(r);
    }
    Landing *L = new (std::nothrow) Landing{s, r};
    if (!L) {
        set_error(FR_ENOMEM, "fractal_server: out of host memory");
        return FR_ENOMEM;
    }
    FR_CUDA(cudaLaunchHostFunc(s->st, on_landed, L));
    return FR_OK;
}

static void worker(fractal_server *s)
{
    cudaSetDevice(s->device);
    std::vector<Request *> admit;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(1), [&] {
                return s->stop || s->error || !s->queue.empty() || !s->resident.empty();
            });
            if (s->error) break;
            if (s->stop && s->queue.empty() && s->resident.empty()) break;
            // admission in arrival order while the budget allows
            admit.clear();
            while (!s->queue.empty()) {
                Request *r = s->queue.front();
                const int64_t need = 2 * (int64_t)al256((size_t)r->f->cells);
                if (s->used + need > s->budget) break;
                s->queue.pop_front();
                s->used += need;
                r->bytes = need;
                admit.push_back(r);
            }
        }
        int rc = FR_OK;
        const double t = now_s();
        for (Request *r : admit) {
            r->t_admit = t;
            const size_t b = al256((size_t)r->f->cells);
            cudaError_t e = cudaMallocAsync((void **)&r->buf[0], 2 * b, s->st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "fractal_server: state allocation");
                break;
            }
            r->buf[1] = r->buf[0] + b;
            rc = fractal_init_bernoulli(r->f, r->buf[0], r->seed, r->p, s->st);
            if (rc) break;
            r->cur = 0;
            r->state = kResident;
            ++s->admitted;
            std::lock_guard<std::mutex> lk(s->mu);
            s->resident.push_back(r);
        }
        if (rc) {
            fail_srv(s, rc, fractal_last_error());
            break;
        }
        std::vector<Request *> active;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request *r : s->resident)
                if (r->remaining > 0) active.push_back(r);
        }
        if (!active.empty()) {
            if (s->gpu_first < 0) s->gpu_first = now_s();
            rc = run_tick(s, active);
            if (rc) {
                fail_srv(s, rc, fractal_last_error());
                break;
            }
        }
        // finished requests leave the resident set and copy their results
        std::vector<Request *> fin;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            auto it = std::stable_partition(s->resident.begin(), s->resident.end(),
                                            [](Request *r) { return r->remaining > 0; });
            fin.assign(it, s->resident.end());
            s->resident.erase(it, s->resident.end());
        }
        for (Request *r : fin) {
            rc = retire(s, r);
            if (rc) break;
        }
        if (rc) {
            fail_srv(s, rc, fractal_last_error());
            break;
        }
    }
}

}  // namespace fr

using namespace fr;

extern "C" int fractal_server_create(int64_t hbm_budget_bytes, int chunk, fractal_server_t **out)
{
    if (!out || chunk < 1) {
        set_error(FR_EINVAL, "fractal_server_create: bad argument");
        return FR_EINVAL;
    }
    fractal_server *s = new (std::nothrow) fractal_server();
    if (!s) {
        set_error(FR_ENOMEM, "fractal_server_create: out of host memory");
        return FR_ENOMEM;
    }
    s->chunk = chunk;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->slots[i].ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&s->pop_ring, sizeof(int64_t) * s->pop_cap);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "fractal_server_create");
    }
    // admission budget: the caller's, capped by 90% of the memory free now
    const int64_t cap = (int64_t)(free_b * 0.9);
    s->budget = (hbm_budget_bytes > 0) ? std::min<int64_t>(hbm_budget_bytes, cap) : cap;
    s->worker = std::thread(worker, s);
    *out = s;
    return FR_OK;
}

extern "C" int fractal_server_submit(fractal_server_t *s, fractal_t *f, uint64_t seed, double p,
                                     int64_t steps, uint32_t birth, uint32_t survive,
                                     uint8_t *host_out, int64_t *id)
{
    if (!s || !f || steps < 0 || !id) {
        set_error(FR_EINVAL, "fractal_server_submit: bad argument");
        return FR_EINVAL;
    }
    // tables are built on the caller's thread, before the worker sees the handle
    int rc = ensure_step_plan(f);
    if (rc) return rc;
    Request *r = new (std::nothrow) Request();
    if (!r) {
        set_error(FR_ENOMEM, "fractal_server_submit: out of host memory");
        return FR_ENOMEM;
    }
    r->f = f;
    r->seed = seed;
    r->p = p;
    r->steps = r->remaining = steps;
    r->birth = birth;
    r->survive = survive;
    r->host_out = host_out;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error) {
            delete r;
            set_error(s->error, "fractal_server_submit: server failed earlier: " + s->error_msg);
            return s->error;
        }
        const int64_t need = 2 * (int64_t)al256((size_t)f->cells);
        if (need > s->budget) {
            delete r;
            set_error(FR_EBUSY, "fractal_server_submit: request larger than the HBM budget");
            return FR_EBUSY;
        }
        r->id = s->next_id++;
        f->server_refs.fetch_add(1);
        s->all[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv.notify_one();
    return FR_OK;
}

// done = 1 when the request's result has landed; latency = completion - submit.
extern "C" int fractal_server_poll(fractal_server_t *s, int64_t id, int *done, double *latency_s,
                                   int64_t *population)
{
    if (!s) {
        set_error(FR_EINVAL, "fractal_server_poll: NULL server");
        return FR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) {
        set_error(FR_ENOTFOUND, "fractal_server_poll: unknown request id");
        return FR_ENOTFOUND;
    }
    const Request *r = it->second;
    if (done) *done = r->state == kDone;
    if (latency_s) *latency_s = (r->state == kDone) ? r->t_done - r->t_submit : -1.0;
    if (population) *population = r->population;
    if (s->error) {
        set_error(s->error, s->error_msg);
        return s->error;
    }
    return FR_OK;
}

extern "C" int fractal_server_wait_all(fractal_server_t *s)
{
    if (!s) {
        set_error(FR_EINVAL, "fractal_server_wait_all: NULL server");
        return FR_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] {
        return s->error || (s->queue.empty() && s->resident.empty() && s->retiring.empty() &&
                            s->completed == s->next_id);
    });
    if (s->error) {
        set_error(s->error, s->error_msg);
        return s->error;
    }
    return FR_OK;
}

extern "C" int fractal_server_stats(fractal_server_t *s, int64_t *completed, int64_t *queued,
                                    int64_t *resident, int64_t *updates, int64_t *launches,
                                    int64_t *hbm_used)
{
    if (!s) {
        set_error(FR_EINVAL, "fractal_server_stats: NULL server");
        return FR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (queued) *queued = (int64_t)s->queue.size();
    if (resident) *resident = (int64_t)s->resident.size();
    if (updates) *updates = s->updates;
    if (launches) *launches = s->launches;
    if (hbm_used) *hbm_used = s->used;
    return FR_OK;
}

extern "C" int fractal_server_destroy(fractal_server_t *s)
{
    if (!s) return FR_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->st);
    for (auto &kv : s->all) {
        Request *r = kv.second;
        if (r->state != kDone) r->f->server_refs.fetch_sub(1);   // a failed server's leftovers
        if (r->buf[0]) cudaFree(r->buf[0]);
        delete r;
    }
    for (auto &u : s->slots) {
        cudaFree(u.dev);
        cudaFreeHost(u.host);
        if (u.ev) cudaEventDestroy(u.ev);
    }
    cudaFreeHost(s->pop_ring);
    cudaStreamDestroy(s->st);
    delete s;
    return FR_OK;
}
