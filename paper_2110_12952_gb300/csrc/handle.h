// handle.h -- the fractal_t handle and the launch plans shared by the .cu
// files of the library (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "internal.cuh"

namespace fr {

// Tables of the bit3 policy (bit3.cuh: 3D, s = 3, tiles of three levels),
// as word offsets into the plan's `pos` array, all copied to shared memory.
struct Bit3Args {
    int k = 0;             // cells per level-1 block (a multiple of 4)
    uint32_t rowset = 0;   // rows dy + 3 dz of a block's 3x3x3 cube that hold members
    int off_rt = 0;        // result bits of row piece (row, 3 bits): 9 x 8 words
    int off_bp = 0;        // block j -> box row of its first row | bit shift << 16: k^2 words
    int off_hs = 0;        // neighbour slot -> its halo entries: first | end << 13 | words needed << 26, 26 words
    int off_he = 0;        // halo entries (two words each, grouped by slot)
    int off_mr = 0;        // members of inner row (y, z) (bits 1..27), 729 words: masks rows of bit states
    int nshared = 0;       // words copied to shared memory
    int off_warp = 0;      // byte offset of warp 0's area in shared memory
    int warp_bytes = 0;    // shared memory per warp (box, pointers, result bits)
    int grid_states = 0;   // blocks per launch of the states -> states generations (smaller shared memory)
    const uint32_t *sin = nullptr;   // multi-generation runs: bit-packed input state (kB3StateWords per tile)
    uint32_t *sout = nullptr;        // and output state, or null
};

// Tiled compact step (Sec. 3 stencil procedure, done per subtree).
// A tile is the k^L cells whose digits above level L agree: one level-L
// subtree, contiguous in omega, whose cells fill an s^L-wide box in the
// embedding.  The local lambda table `pos` (identical for every tile) gives
// each cell's offset in a shared-memory box padded by one halo cell per side.
struct StepPlan {
    int built_levels = -2; // the handle's tile-depth and stage settings the plan was built for
    int built_stages = -2;
    int L = -1;            // tile levels
    int64_t KL = 0;        // k^L cells per tile
    int64_t NT = 0;        // k^(r-L) tiles
    int B = 0;             // s^L, tile box side
    int P = 0;             // B + 2, padded side
    int box_bytes = 0;     // P^dim rounded up to 16
    int coarse_levels = 0; // r - L
    int nring = 0;         // halo cells to fetch per tile
    int nhalo = 0;         // padded-unit policies: runs of halo units copied per tile (ring = their sources)
    int hbytes = 0;        // padded-unit policies: halo bytes copied per tile
    int zoff = 0;          // padded-unit policies: stage offset of the all-zero unit
    uint32_t *pos = nullptr;   // [KL] box offset of local cell l
    uint32_t *ring = nullptr;  // [2*nring] (box offset | slot << 24, local omega)
    int32_t *nbr = nullptr;    // [NT][nbrw] compact index of each neighbour tile, -1 = none
    int nbrw = 0;          // int32 entries per table row (3^dim - 1, padded to 16 B)
    int nstage = 0;        // input pipeline depth
    int stage_bytes = 0;   // one input stage: table row + tile bytes
    int tile_bytes = 0;    // 16-aligned superset of a tile
    int off_bar = 0, off_box = 0, off_pos = 0, off_out = 0;  // shared-memory layout
    int smem = 0;          // dynamic shared memory per CTA
    int block = 256;
    int grid = 0;
    int per_sm = 0;        // resident CTAs per SM
    int mode = 0;          // 0: per-cell neighbour reads; 3 or 4: group mode, block side s^G
    int G = 0;             // levels per group (group mode)
    int KG = 0;            // k^G cells per group
    int Px = 0, Py = 0;    // box row pitch (bytes) and rows per plane
    int ntab = 0;          // entries of the per-tile table (cells or groups)
    int8_t lid_of_q[16] = {};    // block position -> cell of the group, -1 = none
    int16_t rel_of_lid[16] = {}; // cell of the group -> offset from the window base
    int xoff = 0;                // box byte of padded column 0 (3 in quad mode)
    int tapz = 0;                // tap mode: index of the all-zero group
    int nq = 0;                  // tap mode: units per tile
    uint32_t row_sel[8] = {};    // quad mode: byte selectors, group cells -> block rows
    uint32_t pack_sel[9] = {};   // quad mode: byte selectors, block sums -> cell order
    Bit3Args b3;                 // bit3 mode
};

// Bounding-box step (Sec. 4 "BB"): membership of a box cell is decided from
// two bitmaps, the lowest Lb levels (local) and the levels above (coarse).
struct BBPlan {
    int Lb = -1;
    int S = 0;             // s^Lb, local side
    int C = 0;             // s^(r-Lb), coarse side
    uint32_t *local_bits = nullptr;   // S^dim bits, x fastest
    uint32_t *coarse_bits = nullptr;  // C^dim bits, x fastest
    int64_t local_words = 0, coarse_words = 0;
};

// Temporal blocking (temporal.cuh): tile depth, tables and launch shape of
// the multi-generation pass for the carpet and the Vicsek fractal.
struct TbPlan {
    int L = -1;
    int preset = -1;
    int64_t KL = 0, NT = 0;
    int nu = 0, nring = 0, W = 0, RS = 0, NWB = 0;
    int off_halo = 0, off_pres = 0, off_box0 = 0, off_box1 = 0, off_mask = 0;
    int smem = 0, block = 0, grid = 0, per_sm = 0;
    uint16_t *upos = nullptr;
    uint32_t *ring = nullptr;
    int32_t *nbr = nullptr;
};

// fractal_run_host's pipeline for one generation: the tiles in chunks
// (omega order), each chunk computed once the chunks that hold its tiles'
// neighbours have arrived, its results copied back while later chunks are
// still arriving.
struct HostPipe {
    int L = -1;
    int64_t NT = 0;
    std::vector<int64_t> bounds;   // chunk c = tiles bounds[c] .. bounds[c+1] - 1
    std::vector<int> need;         // the last input chunk chunk c reads
    std::vector<int> order;        // chunks by need, then index
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_out;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

}  // namespace fr

struct fractal {
    int k = 0, s = 0, r = 0, dim = 0;
    std::vector<int32_t> offsets;
    int64_t cells = 0;     // k^r
    int64_t side = 0;      // s^r
    int64_t box_cells = 0; // side^dim, or -1 when it overflows int64
    fr::FracDev dev{};
    int device = 0;
    int num_sms = 0;
    int tile_levels_user = -1;
    int stages_user = -1;            // input pipeline stages (2..4), -1 = the policy's default
    fr::StepPlan plan;
    fr::BBPlan bb;
    uint8_t *scratch = nullptr;      // k^r bytes, ping-pong for steps > 1
    uint32_t *b3_state[2] = {nullptr, nullptr};  // bit3 plans, steps > 1: bit-packed tile states (ping-pong)
    uint8_t *bb_scratch = nullptr;   // n^dim bytes, ping-pong for BB steps > 1
    uint8_t *host_io[2] = {nullptr, nullptr};  // device buffers of run_host
    fr::HostPipe pipe;                          // run_host's chunked pipeline
    int *status = nullptr;           // device word set by kernels whose bounded waits gave up
    std::atomic<int> server_refs{0}; // requests of a server not yet done (the plan must not change)
    int tb_gens = 0;                 // temporal blocking: generations per pass (0 = off)
    int tb_levels_user = -1;         // its tile depth (-1 = automatic)
    fr::TbPlan tb;
    void *paper_aux = nullptr;       // the paper's approaches (paper_kernels.cu): geometry and scratch
    // a different transition table per level (fractal_create_mixed); then
    // `offsets` holds the levels' tables one after the other
    bool mixed = false;
    std::vector<int32_t> lev_k;              // replica count of each level
    std::vector<int64_t> lev_first;          // first offset row of each level's table
    std::vector<std::vector<int16_t>> lev_hinv;   // digit tuple -> replica, per level
    fr::MixLevel *d_mix = nullptr;           // the same in device memory
    uint32_t test_extra_tx = 0;      // fractal_test_arm_timeout: next step launch's extra armed bytes
    uint32_t test_wait_limit = 0;    // ... and its wait limit (tries)
};

namespace fr {

// cells of a level-L subtree (product of the replica counts of levels
// 0 .. L-1) and subtrees of level L (levels L .. r-1)
inline int64_t cells_below(const fractal *f, int L)
{
    int64_t v = 1;
    for (int mu = 0; mu < L; ++mu) v *= f->mixed ? f->lev_k[mu] : f->k;
    return v;
}
inline int64_t cells_above(const fractal *f, int L)
{
    int64_t v = 1;
    for (int mu = L; mu < f->r; ++mu) v *= f->mixed ? f->lev_k[mu] : f->k;
    return v;
}

int ensure_step_plan(fractal *f);
int ensure_tb_plan(fractal *f);
void fr_paper_aux_free(fractal *f);
void free_tb_plan(TbPlan &p);
int launch_tb_once(fractal *f, const uint8_t *in, uint8_t *out, int gens, uint32_t birth, uint32_t survive,
                   cudaStream_t st);
int ensure_bb_plan(fractal *f);
void free_step_plan(StepPlan &p);
void free_bb_plan(BBPlan &p);

int launch_step_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                     uint32_t survive, cudaStream_t st);
// One generation of the instance's tiles T0 .. T1 - 1 only (the others are
// read as neighbours, not written).
int launch_step_range(fractal *f, const uint8_t *in, uint8_t *out, int64_t T0, int64_t T1, uint32_t birth,
                      uint32_t survive, cudaStream_t st);
// Whether the handle's step plan is the bit3 policy; `steps` >= 2
// generations of such a plan with the state bit-packed between them (the
// first generation reads bytes, the last writes them).
bool bit3_plan(const fractal *f);
int launch_bit3_generations(fractal *f, const uint8_t *in, uint8_t *out, int64_t steps, uint32_t birth,
                            uint32_t survive, cudaStream_t st);
// One generation of the tiles 0 .. ntiles-1 of the buffer `in` (tile T at
// cell T k^L) with the neighbour table `nbr` (ntiles rows, indices of tiles
// of the same buffer, which holds readable_cells cells), into `out`.
int launch_step_tiles(fractal *f, const uint8_t *in, uint8_t *out, const int32_t *nbr, int64_t ntiles,
                      int64_t readable_cells, uint32_t birth, uint32_t survive, cudaStream_t st);
int launch_bb_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                   uint32_t survive, cudaStream_t st);
int launch_copy_normalise(const uint8_t *in, uint8_t *out, int64_t n, int num_sms, cudaStream_t st);
int preload_copy_kernel();
int ensure_status(fractal *f);
int take_status(fractal *f);
int cached_tile_levels(const fractal *f, int *stages);
int autotune_step(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth, uint32_t survive,
                  cudaStream_t st, int *best);

}  // namespace fr
