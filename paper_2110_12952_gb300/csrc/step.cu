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
//     halo.  Cells of the box that are not local members stay 0; halo cells
//     that are members and touch a member of the tile (list `ring`) are
//     fetched from the neighbouring tiles.
//
// Three ways to count neighbours from the box (the "policy" of the kernel):
//   * quad (2D, s = 2, k = 3): a level-2 group is 9 cells, contiguous in
//     omega, filling a 4x4 block.  A thread owns 4 consecutive groups (36
//     bytes = 9 aligned words of input and of output).  Box rows of a block
//     are assembled with byte permutes and stored as words; the 6x6 window of
//     a block is added byte-wise (a byte holds a count <= 9, so no carry
//     crosses a byte): three row adds give vertical sums, two funnel shifts
//     and two adds give the 3x3 sums of a block row.  The sums are permuted
//     back into omega order and the rule is applied to 4 cells at a time as a
//     byte look-up (prmt).
//   * group (2D, s^G = 3 or 4): the same window sums per group, one thread
//     per group, byte stores.
//   * cell (any other case, 3D): each cell reads its 3^dim - 1 neighbours.
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "handle.h"
#include "step.h"
#include "tma.cuh"
#include "rows_layout.h"
#include "lid_layout.h"
#include "bit3_layout.h"

namespace fr {

constexpr int kMaxGroup = 16;  // cells per group / block positions (s^G <= 4)
constexpr int kQuadKG = 9;     // cells per group in quad mode
constexpr int kRingRegs = 4;   // halo values per thread prefetched in registers
constexpr int kRunGap = 2;     // padded units: unneeded units a halo run may span
constexpr int kRunMax = 8;     // padded units: most units per halo run

struct StepArgs {
    int64_t KL, NT, cells;
    int64_t tile0;         // single-instance launches: the first tile of the launch (tiles tile0 .. tile0 + NT - 1)
    int Px, Py;            // box row pitch and rows per plane (bytes / rows)
    int nring, nbrw, nstage, stage_bytes, tile_bytes;
    int nhalo;             // padded-unit policies: runs of halo units per tile, in `ring`
    int hbytes, zoff;      // padded-unit policies: halo bytes per tile, zero unit's stage offset
    int off_bar, off_box, off_tab, off_out, box_bytes;
    int ntab;              // entries of the shared table (cells or groups)
    int KG;                // cells per group (group / quad mode)
    int tapz;              // tap mode: byte offset of the all-zero group; unit policies: its index
    int nq;                // tap mode: units per tile
    uint32_t wait_limit;   // tries of each bounded wait (kWaitLimit unless a test shortened it)
    uint32_t extra_tx;     // bytes each stage is armed for beyond its copies (0 unless a test set it)
    const uint32_t *tab;   // cell mode: box offset per cell; else window base per group
    const uint32_t *ring;
    const int32_t *nbr;
    Rule rule;             // single-instance launches
    int *status;
    // multi-instance launches (tile_inst != nullptr)
    const int32_t *tile_inst;
    const InstDesc *insts;
    int gen;
    int8_t lid_of_q[kMaxGroup];     // block position -> cell of the group, -1 none
    int16_t rel_of_lid[kMaxGroup];  // cell of the group -> box offset from the window base
    uint32_t row_sel[8];            // quad: cells -> block row j (two selectors per row)
    uint32_t pack_sel[9];           // quad: block sums -> cell order (three per word)
    Bit3Args b3;                    // bit3 policy: its tables in `tab`
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
    if (f->mixed) {
        for (int mu = 0; mu < L; ++mu) {
            const int k = f->lev_k[mu];
            const int d = (int)(l % k);
            l /= k;
            const int32_t *off = f->offsets.data() + (f->lev_first[mu] + d) * f->dim;
            for (int i = 0; i < f->dim; ++i) p[i] += (int)(sm * off[i]);
            sm *= f->s;
        }
        return;
    }
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
        const int h = f->mixed ? f->lev_hinv[mu][t] : f->dev.hinv[t];
        if (h < 0) return -1;
        w += h * km;
        km *= f->mixed ? f->lev_k[mu] : f->k;
    }
    return w;
}

static int nbr_width(int dim) { return dim == 3 ? 28 : 8; }  // 26 or 8 entries, 16-byte rows

// ---- bit3 mode (3D fractals with s = 3, see bit3.cuh): tiles of three
// levels, level-1 blocks of k bytes read as k / 4 words
static bool bit3_ok(const fractal *f, int L)
{
    return f->dim == 3 && f->s == 3 && !f->mixed && L == 3 && f->r >= 3 && f->k % 4 == 0 && f->k <= 24;
}

// halo entries of a 3D fractal with s = 3 at three levels: per neighbour
// direction, the blocks of that tile which touch the box's one-cell ring,
// and (in hs) the words of a block that hold the cells those blocks
// contribute (the same for every block of a direction)
static std::vector<uint32_t> bit3_halo(const fractal *f, std::vector<uint32_t> &hs)
{
    std::vector<uint32_t> he;
    hs.assign(26, 0u);
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        const int dir[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
        const int slot = q < 13 ? q : q - 1;
        const uint32_t first = (uint32_t)(he.size() / 2);
        uint32_t words = 0;
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = dir[a] < 0 ? 8 : 0;   // the neighbour's blocks next to this tile
            hi[a] = dir[a] > 0 ? 0 : 8;
        }
        for (int bz = lo[2]; bz <= hi[2]; ++bz)
            for (int by = lo[1]; by <= hi[1]; ++by)
                for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                    const int c[3] = {bx, by, bz};
                    const int64_t jb = host_nu(f, c, 2);
                    if (jb < 0) continue;
                    // box coordinates of the block's first cell (the box's
                    // interior is 1 .. 27, its ring 0 and 28)
                    const int o[3] = {1 + 27 * dir[0] + 3 * bx, 1 + 27 * dir[1] + 3 * by, 1 + 27 * dir[2] + 3 * bz};
                    uint32_t rmask = 0, pmask = 0;
                    for (int rr = 0; rr < 9; ++rr) {
                        const int y = o[1] + rr % 3, z = o[2] + rr / 3;
                        if (y >= 0 && y <= 28 && z >= 0 && z <= 28) rmask |= 1u << rr;
                    }
                    for (int x0 = 0; x0 < 3; ++x0)
                        if (o[0] + x0 >= 0 && o[0] + x0 <= 28) pmask |= 1u << x0;
                    for (int rr = 0; rr < 9; ++rr)
                        for (int x0 = 0; x0 < 3; ++x0) {
                            const int h = f->dev.hinv[x0 + 3 * rr];
                            if (((rmask >> rr) & 1) && ((pmask >> x0) & 1) && h >= 0) words |= 1u << (h / 4);
                        }
                    const int rowbase = o[1] + kB3Pitch * o[2];
                    he.push_back((uint32_t)slot | (uint32_t)jb << 5 | rmask << 15 | pmask << 24 |
                                 (uint32_t)(o[0] + 2) << 27);
                    he.push_back((uint32_t)rowbase);
                }
        hs[slot] = first | (uint32_t)(he.size() / 2) << 13 | words << 26;
    }
    return he;
}

static int bit3_shared_words(const fractal *f)
{
    std::vector<uint32_t> hs;
    const size_t nhe = bit3_halo(f, hs).size();
    return (int)((f->k / 4) * 16 + 72 + f->k * f->k + 26 + 2 + nhe + 729);
}
static int bit3_warp_bytes(const fractal *f) { return kB3OffBits + (int)round16(((int64_t)f->k * f->k * f->k + 7) / 8); }

// The bit3 tables, in the order of Bit3Args: cube bits of each nibble of
// each word of a block; result bits of each 3-bit row piece; box row and bit
// shift of each block of a tile; the halo entries by neighbour slot; the
// member bits of each inner box row.  A halo
// entry is slot | block index << 5 | rows in the ring << 15 | cells of a row
// piece in the ring << 24 | (box bit of the piece's first cell + 2) << 27,
// then the box row of the block's first row (which may lie outside the box).
static std::vector<uint32_t> bit3_tables(const fractal *f, Bit3Args &b)
{
    const int k = f->k, kw = k / 4;
    std::vector<uint32_t> t;
    b.k = k;
    for (int q = 0; q < kw; ++q)
        for (int nib = 0; nib < 16; ++nib) {
            uint32_t m = 0;
            for (int i = 0; i < 4; ++i)
                if ((nib >> i) & 1) {
                    const int32_t *o = &f->offsets[(size_t)(4 * q + i) * 3];
                    m |= 1u << (o[0] + 3 * o[1] + 9 * o[2]);
                }
            t.push_back(m);
        }
    b.off_rt = (int)t.size();
    b.rowset = 0;
    for (int rr = 0; rr < 9; ++rr)             // row rr = dy + 3 dz of the cube
        for (int piece = 0; piece < 8; ++piece) {
            uint32_t m = 0;
            for (int x = 0; x < 3; ++x) {
                const int h = f->dev.hinv[x + 3 * rr];
                if (h >= 0) b.rowset |= 1u << rr;
                if (h >= 0 && ((piece >> x) & 1)) m |= 1u << h;
            }
            t.push_back(m);
        }
    b.off_bp = (int)t.size();
    for (int j = 0; j < k * k; ++j) {
        int c[3];
        host_lambda(f, j, 2, c);   // block j of a tile: its place in the 9^3 grid of blocks
        const int rb = (1 + 3 * c[1]) + kB3Pitch * (1 + 3 * c[2]);
        t.push_back((uint32_t)rb | (uint32_t)(1 + 3 * c[0]) << 16);
    }
    std::vector<uint32_t> hs;
    const std::vector<uint32_t> he = bit3_halo(f, hs);
    b.off_hs = (int)t.size();
    t.insert(t.end(), hs.begin(), hs.end());
    while (t.size() % 2) t.push_back(0);
    b.off_he = (int)t.size();
    t.insert(t.end(), he.begin(), he.end());
    b.off_mr = (int)t.size();
    for (int z = 0; z < 27; ++z)
        for (int y = 0; y < 27; ++y) {
            uint32_t m = 0;
            for (int x = 0; x < 27; ++x) {
                const int c[3] = {x, y, z};
                if (host_nu(f, c, 3) >= 0) m |= 1u << (x + 1);
            }
            t.push_back(m);
        }
    b.nshared = (int)t.size();
    return t;
}
static int nstages() { return 3; }

// Group mode applies to 2D fractals whose block side s^G is 3 or 4.
static int group_levels(const fractal *f)
{
    if (f->dim != 2 || f->mixed) return 0;
    if (f->s == 2) return 2;
    if (f->s == 3 || f->s == 4) return 1;
    return 0;
}

enum { kModeCell = 0, kModeGroup3 = 3, kModeGroup4 = 4, kModeQuad = 9, kModeTap = 10, kModeRows0 = 11, kModeRows1 = 12, kModeLid1 = 13,
       kModeBox3 = 14, kModeBit3 = 15 };

// ---- box3 mode (3D fractals, see box3.cuh): box row pitch, a multiple of
// 16 bytes with at least one zero word after the B + 2 padded cells
static int64_t box3_pitch(int64_t B)
{
    return (4 * ((B + 3) / 4) + 4 + 15) / 16 * 16;
}

// ---- tap mode: the Sierpinski triangle with offsets (0,0), (1,0), (0,1)
// A level-2 group is 9 cells (lid 0..8 at kPosX/kPosY) filling a 4x4 block.
// The 6x6 window of a block needs, besides its own cells, only 8 border
// cells ("taps") that are members of a neighbouring block and touch a
// member of the block.  They come from 6 neighbouring groups, in the order
// W, E, N, NE, S, SW.
constexpr int kTapDirs = 6;
constexpr int kTapDx[kTapDirs] = {-1, 1, 0, 1, 0, -1};
constexpr int kTapDy[kTapDirs] = {0, 0, -1, -1, 1, 1};
constexpr int kTaps = 8;
// dir index, lid in that neighbour, window row, window column (0..5); in
// the order W4 E0 E2 N8 NE8 S0 S1 SW4 (direction, then lid)
constexpr int kTap[kTaps][4] = {{0, 4, 1, 0}, {1, 0, 1, 5}, {1, 2, 2, 5}, {2, 8, 0, 1},
                                {3, 8, 0, 5}, {4, 0, 5, 1}, {4, 1, 5, 2}, {5, 4, 5, 0}};
static const int32_t kTriangleOffsets[6] = {0, 0, 1, 0, 0, 1};

// A thread owns a unit: 9 consecutive groups (81 cells, a level-4 subtree),
// whose groups sit in the 4x4 block of groups at the same positions as the
// cells of a group in its block (two base-3 digits each picking offset
// (0,0), (1,0) or (0,1) at its scale).
constexpr int kUnitGroups = 9;
constexpr int kUnitCells = 81;
constexpr int kPosX[9] = {0, 1, 0, 2, 3, 2, 0, 1, 0};
constexpr int kPosY[9] = {0, 0, 1, 0, 0, 1, 2, 2, 3};
// The 12 groups around a unit that its taps read (position relative to the
// unit's first group, in groups) and the 14 tap cells in them.
constexpr int kExtGroups = 12;
constexpr int kExtDx[kExtGroups] = {0, 1, 2, 3, 4, 4, -1, -1, -1, -1, -1, 0};
constexpr int kExtDy[kExtGroups] = {-1, -1, -1, -1, -1, 0, 0, 1, 2, 3, 4, 4};
constexpr int kExtCells = 14;
constexpr int kXg[kExtCells] = {0, 1, 2, 3, 4, 5, 5, 6, 7, 8, 9, 10, 11, 11};
constexpr int kXlid[kExtCells] = {8, 8, 8, 8, 8, 0, 2, 4, 4, 4, 4, 4, 0, 1};
constexpr int kSrcZero = -1, kSrcBad = -2, kSrcExt = 1000;
constexpr int kTapHaloGap = 16;   // bytes between a tile's last cell and its first halo group

// Source of tap t of group j of a unit: byte 9 j' + lid of the unit (a
// group of the same unit), kSrcZero (a hole of the unit's block) or
// kSrcExt + c (external tap cell c).
constexpr int tap_src(int j, int t)
{
    const int nx = kPosX[j] + kTapDx[kTap[t][0]], ny = kPosY[j] + kTapDy[kTap[t][0]];
    const int lid = kTap[t][1];
    if (nx >= 0 && nx < 4 && ny >= 0 && ny < 4) {
        for (int g = 0; g < kUnitGroups; ++g)
            if (kPosX[g] == nx && kPosY[g] == ny) return 9 * g + lid;
        return kSrcZero;
    }
    for (int c = 0; c < kExtCells; ++c)
        if (kExtDx[kXg[c]] == nx && kExtDy[kXg[c]] == ny && kXlid[c] == lid) return kSrcExt + c;
    return kSrcBad;
}

constexpr bool unit_taps_resolved()
{
    for (int j = 0; j < kUnitGroups; ++j)
        for (int t = 0; t < kTaps; ++t)
            if (tap_src(j, t) == kSrcBad) return false;
    return true;
}
static_assert(unit_taps_resolved(), "every tap outside a unit's block is one of its external cells");

static bool is_triangle(const fractal *f)
{
    if (f->mixed || f->dim != 2 || f->s != 2 || f->k != 3) return false;
    for (int i = 0; i < 6; ++i)
        if (f->offsets[i] != kTriangleOffsets[i]) return false;
    return true;
}

// Tables of tap mode for tile depth L (4 <= L): per unit, the byte offsets
// 9 g (uint16, two per word) of its 12 external groups from the tile's
// first cell in the stage, where halo groups continue after the tile's NG
// groups and group NG + H is all zero; and the halo bytes to fetch per tile
// (ring entries: byte offset from the tile's first cell in the stage |
// tile-table slot << 24, cell offset in the neighbouring tile).
struct TapTables {
    int NG = 0, NQ = 0, H = 0;
    int zero_off = 0;              // byte offset of the all-zero group from the tile's first cell
    std::vector<uint32_t> words;   // NQ * 6
    std::vector<uint32_t> ring;
    bool ok = false;
};

static void host_lambda(const fractal *f, int64_t l, int L, int p[3]);
static int64_t host_nu(const fractal *f, const int q[3], int L);

static TapTables tap_tables(const fractal *f, int L)
{
    TapTables t;
    if (!is_triangle(f) || L < 4) return t;
    const int NB = 1 << (L - 2);            // blocks per side
    int NG = 1;
    for (int i = 0; i < L - 2; ++i) NG *= 3;
    t.NG = NG;
    t.NQ = NG / kUnitGroups;
    std::vector<int> M((size_t)NB * NB, -1);
    std::vector<int> bx(NG), by(NG);
    for (int g = 0; g < NG; ++g) {
        int c[3];
        host_lambda(f, g, L - 2, c);
        bx[g] = c[0];
        by[g] = c[1];
        M[(size_t)c[1] * NB + c[0]] = g;
    }
    // the cell layout of a group and the group layout of a unit
    for (int lid = 0; lid < 9; ++lid) {
        int c[3];
        host_lambda(f, lid, 2, c);
        if (c[0] != kPosX[lid] || c[1] != kPosY[lid]) return t;
    }
    for (int g = 0; g < NG; ++g) {
        const int g0 = g - g % kUnitGroups;
        if (bx[g] != bx[g0] + kPosX[g % kUnitGroups] || by[g] != by[g0] + kPosY[g % kUnitGroups]) return t;
    }
    // check the constant tap list against the fractal: every border cell of
    // a window that is a member and touches a member of the block is a tap
    {
        int lid_of[4][4];
        for (int y = 0; y < 4; ++y)
            for (int x = 0; x < 4; ++x) {
                int q[3] = {x, y, 0};
                lid_of[y][x] = (int)host_nu(f, q, 2);
            }
        int found = 0;
        for (int wr = 0; wr < 6; ++wr)
            for (int wc = 0; wc < 6; ++wc) {
                if (wr >= 1 && wr <= 4 && wc >= 1 && wc <= 4) continue;
                const int x = wc - 1, y = wr - 1;
                const int dx = x < 0 ? -1 : (x > 3 ? 1 : 0), dy = y < 0 ? -1 : (y > 3 ? 1 : 0);
                const int lid = lid_of[(y + 4) % 4][(x + 4) % 4];
                bool touch = false;
                for (int ey = -1; ey <= 1; ++ey)
                    for (int ex = -1; ex <= 1; ++ex) {
                        const int ax = x + ex, ay = y + ey;
                        if (ax >= 0 && ax < 4 && ay >= 0 && ay < 4 && lid_of[ay][ax] >= 0) touch = true;
                    }
                if (lid < 0 || !touch) continue;
                bool listed = false;
                for (int k = 0; k < kTaps; ++k)
                    if (kTapDx[kTap[k][0]] == dx && kTapDy[kTap[k][0]] == dy && kTap[k][1] == lid &&
                        kTap[k][2] == wr && kTap[k][3] == wc)
                        listed = true;
                if (!listed) return t;
                ++found;
            }
        if (found != kTaps) return t;
        // rule4_sparse: no member has more than 6 member neighbours (the
        // block's members and the taps are every member its cells touch)
        int win[6][6] = {};
        for (int lid = 0; lid < 9; ++lid) win[kPosY[lid] + 1][kPosX[lid] + 1] = 1;
        for (int k = 0; k < kTaps; ++k) win[kTap[k][2]][kTap[k][3]] = 1;
        for (int lid = 0; lid < 9; ++lid) {
            int n = 0;
            for (int ey = -1; ey <= 1; ++ey)
                for (int ex = -1; ex <= 1; ++ex)
                    if (ex || ey) n += win[kPosY[lid] + 1 + ey][kPosX[lid] + 1 + ex];
            if (n > 6) return t;
        }
    }
    uint32_t ext_lids[kExtGroups] = {};
    for (int c = 0; c < kExtCells; ++c) ext_lids[kXg[c]] |= 1u << kXlid[c];
    // external groups of every unit; halo slots for groups of neighbouring tiles
    std::map<std::pair<int, int>, int> slot_of;   // (tile-table slot, group there) -> halo slot
    std::vector<std::pair<int, int>> slots;
    std::vector<uint32_t> lids_read;               // per halo slot: mask of the lids some tap reads
    std::vector<int> ext((size_t)t.NQ * kExtGroups);
    for (int q = 0; q < t.NQ; ++q)
        for (int e = 0; e < kExtGroups; ++e) {
            int nx = bx[kUnitGroups * q] + kExtDx[e], ny = by[kUnitGroups * q] + kExtDy[e];
            const int tdx = nx < 0 ? -1 : (nx >= NB ? 1 : 0), tdy = ny < 0 ? -1 : (ny >= NB ? 1 : 0);
            nx = (nx + NB) % NB;
            ny = (ny + NB) % NB;
            const int gn = M[(size_t)ny * NB + nx];
            int v = -2;                               // -2: the zero group
            if (gn >= 0) {
                if (tdx == 0 && tdy == 0) v = gn;
                else {
                    const int dir9 = (tdx + 1) + 3 * (tdy + 1);
                    const int tslot = dir9 < 4 ? dir9 : dir9 - 1;
                    auto key = std::make_pair(tslot, gn);
                    auto it = slot_of.find(key);
                    if (it == slot_of.end()) {
                        it = slot_of.emplace(key, (int)slots.size()).first;
                        slots.push_back(key);
                        lids_read.push_back(0);
                    }
                    lids_read[it->second] |= ext_lids[e];
                    v = -100 - it->second;            // halo slot, resolved below
                }
            }
            ext[(size_t)q * kExtGroups + e] = v;
        }
    t.H = (int)slots.size();
    // halo group hs sits kTapHaloGap bytes past the tile's last cell (out of
    // reach of the tile's 16-byte-rounded bulk copy, so that its plain
    // stores never race the copy), the zero group after the halo groups
    auto halo_off = [&](int hs) { return 9 * NG + kTapHaloGap + 9 * hs; };
    t.zero_off = halo_off(t.H);
    if (t.zero_off + 8 >= 65536) return t;
    t.words.assign((size_t)t.NQ * kExtGroups / 2, 0);
    for (int q = 0; q < t.NQ; ++q)
        for (int e = 0; e < kExtGroups; ++e) {
            const int v = ext[(size_t)q * kExtGroups + e];
            const uint32_t b = (v == -2) ? (uint32_t)t.zero_off
                                         : (v <= -100 ? (uint32_t)halo_off(-100 - v) : 9u * (uint32_t)v);
            t.words[(size_t)q * (kExtGroups / 2) + e / 2] |= b << (16 * (e % 2));
        }
    // only the halo cells that a tap reads are staged; the other bytes of a
    // halo group are never read
    for (int hs = 0; hs < t.H; ++hs)
        for (int lid = 0; lid < 9; ++lid) {
            if (!((lids_read[hs] >> lid) & 1u)) continue;
            t.ring.push_back((uint32_t)(halo_off(hs) + lid) | ((uint32_t)slots[hs].first << 24));
            t.ring.push_back((uint32_t)(9 * slots[hs].second + lid));
        }
    if (t.ring.size() / 2 > 32) return t;   // one halo cell per lane of the refilling warp
    t.ok = true;
    return t;
}

// ---- rows mode: the carpet and the Vicsek fractal (see rows_layout.h)
static int rows_preset_of(const fractal *f)
{
    if (f->mixed || f->dim != 2 || f->s != 3) return -1;
    auto same = [&](int k, const int *ox, const int *oy) {
        if (f->k != k) return false;
        for (int j = 0; j < k; ++j)
            if (f->offsets[2 * j] != ox[j] || f->offsets[2 * j + 1] != oy[j]) return false;
        return true;
    };
    if (same(RowsPreset<0>::k, RowsPreset<0>::ox, RowsPreset<0>::oy)) return 0;
    if (same(RowsPreset<1>::k, RowsPreset<1>::ox, RowsPreset<1>::oy)) return 1;
    return -1;
}

// Tables of rows mode for tile depth L (>= 2): per unit (level-2 subtree of
// the tile), the byte offsets (uint16, two per word) of its 8 neighbouring
// units in the order of frame_dir, from the tile's first cell in the stage:
// units of the tile at slot u (rp_slot), halo units of neighbouring tiles
// after them, then an all-zero unit; and the halo bytes to fetch per tile
// (ring entries as in tap mode), or for padded units the runs of halo units
// to copy whole.
struct RowsTables {
    int NU = 0, H = 0;
    std::vector<uint32_t> words;   // NU * 4
    std::vector<uint32_t> ring;    // contiguous units: halo cells (ring entries)
    // padded units: per run of halo units, (tile-table slot << 24 | first
    // unit, stage offset << 8 | units)
    std::vector<uint32_t> halo;
    int hbytes = 0;                // padded units: halo bytes per tile
    int zoff = 0;                  // stage offset of the zero unit
    int64_t data_bytes = 0;        // padded units: stage data bytes
    bool ok = false;
};

template <int P>
static RowsTables rows_tables(const fractal *f, int L)
{
    RowsTables t;
    constexpr int K = RowsPreset<P>::k, NB = K * K;
    if (rows_preset_of(f) != P || L < 2) return t;
    int side = 1, NU = 1;
    for (int i = 0; i < L - 2; ++i) {
        side *= 3;
        NU *= K;
    }
    t.NU = NU;
    std::vector<int> M((size_t)side * side, -1);
    std::vector<int> ux(NU), uy(NU);
    for (int q = 0; q < NU; ++q) {
        int c[3];
        host_lambda(f, q, L - 2, c);
        ux[q] = c[0];
        uy[q] = c[1];
        M[(size_t)c[1] * side + c[0]] = q;
    }
    // the unit layout against the fractal's own lambda
    for (int q = 0; q < NU; ++q)
        for (int u = 0; u < NB; ++u) {
            int c[3];
            host_lambda(f, (int64_t)NB * q + u, L, c);
            if (c[0] != 9 * ux[q] + rp_x<P>(u) || c[1] != 9 * uy[q] + rp_y<P>(u)) return t;
        }
    uint64_t dir_bytes[8] = {};   // per direction: the unit bytes some frame cell reads
    for (int fr = 0; fr < kFrame; ++fr)
        if (frame_byte<P>(fr) >= 0) dir_bytes[frame_dir(fr)] |= 1ull << frame_byte<P>(fr);
    std::map<std::pair<int, int>, int> slot_of;   // (tile-table slot, unit there) -> halo unit
    std::vector<std::pair<int, int>> slots;
    std::vector<uint64_t> bytes_read;
    std::vector<int> nb((size_t)NU * 8);
    for (int q = 0; q < NU; ++q)
        for (int d = 0; d < 8; ++d) {
            const int d9 = d < 4 ? d : d + 1;
            int nx = ux[q] + d9 % 3 - 1, ny = uy[q] + d9 / 3 - 1;
            const int tdx = nx < 0 ? -1 : (nx >= side ? 1 : 0), tdy = ny < 0 ? -1 : (ny >= side ? 1 : 0);
            nx = (nx + side) % side;
            ny = (ny + side) % side;
            const int gn = M[(size_t)ny * side + nx];
            int v = -2;   // -2: the zero unit
            if (gn >= 0 && dir_bytes[d]) {
                if (tdx == 0 && tdy == 0) v = gn;
                else {
                    const int t9 = (tdx + 1) + 3 * (tdy + 1);
                    const int tslot = t9 < 4 ? t9 : t9 - 1;
                    auto key = std::make_pair(tslot, gn);
                    auto it = slot_of.find(key);
                    if (it == slot_of.end()) {
                        it = slot_of.emplace(key, (int)slots.size()).first;
                        slots.push_back(key);
                        bytes_read.push_back(0);
                    }
                    bytes_read[it->second] |= dir_bytes[d];
                    v = -100 - it->second;
                }
            }
            nb[(size_t)q * 8 + d] = v;
        }
    t.H = (int)slots.size();
    // stage byte offsets of the halo units and of the zero unit
    std::vector<int> hoff(t.H);
    int zoff;
    if constexpr (rp_padded<P>()) {
        // halo units copied whole, in runs: per neighbouring tile, its
        // needed units in increasing order, one run spanning gaps of at most
        // kRunGap unneeded units and at most kRunMax units, the runs back to
        // back (unpadded: only byte loads read them) after the tile's units
        std::vector<int> order(t.H);
        for (int h = 0; h < t.H; ++h) order[h] = h;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return slots[x] < slots[y]; });
        const int hb = rp_slot<P>(NU);
        int pos = hb;
        for (int i = 0; i < t.H;) {
            const int ts = slots[order[i]].first, first = slots[order[i]].second;
            int last = first, j = i + 1;
            while (j < t.H && slots[order[j]].first == ts && slots[order[j]].second - last <= kRunGap + 1 &&
                   slots[order[j]].second - first < kRunMax)
                last = slots[order[j++]].second;
            for (int m = i; m < j; ++m) hoff[order[m]] = pos + NB * (slots[order[m]].second - first);
            t.halo.push_back((uint32_t)first | ((uint32_t)ts << 24));
            t.halo.push_back(((uint32_t)pos << 8) | (uint32_t)(last - first + 1));
            pos += NB * (last - first + 1);
            i = j;
        }
        t.hbytes = pos - hb;
        zoff = pos;
        t.data_bytes = zoff + NB;
    } else {
        for (int h = 0; h < t.H; ++h) hoff[h] = rp_slot<P>(NU + h);
        zoff = rp_slot<P>(NU + t.H);
    }
    if ((int64_t)zoff + NB >= 65536) return t;
    t.zoff = zoff;
    t.words.assign((size_t)NU * 4, 0);
    for (int q = 0; q < NU; ++q)
        for (int d = 0; d < 8; ++d) {
            const int v = nb[(size_t)q * 8 + d];
            const uint32_t off = (uint32_t)(v == -2 ? zoff : (v <= -100 ? hoff[-100 - v] : rp_slot<P>(v)));
            t.words[(size_t)q * 4 + d / 2] |= off << (16 * (d % 2));
        }
    // contiguous units: only the halo bytes some frame cell reads are staged
    if constexpr (!rp_padded<P>()) {
        for (int hs = 0; hs < t.H; ++hs)
            for (int b = 0; b < NB; ++b) {
                if (!((bytes_read[hs] >> b) & 1u)) continue;
                t.ring.push_back((uint32_t)(hoff[hs] + b) | ((uint32_t)slots[hs].first << 24));
                t.ring.push_back((uint32_t)(NB * slots[hs].second + b));
            }
    }
    t.ok = true;
    return t;
}

// ---- lid mode: the Vicsek fractal in level-3 units (see lid_layout.h)
constexpr int kLidPreset = 1, kLidLevels = 3;

// Tables of lid mode for tile depth L (>= kLidLevels), laid out as those of
// rows mode with units of k^3 cells (27x27 blocks).
template <int P, int U>
static RowsTables lid_tables(const fractal *f, int L)
{
    RowsTables t;
    constexpr int NB = LidUnit<P, U>::NB, SIDE = LidUnit<P, U>::side, NE = lu_next<P, U>();
    if (rows_preset_of(f) != P || L < U) return t;
    int side = 1, NU = 1;
    for (int i = 0; i < L - U; ++i) {
        side *= 3;
        NU *= RowsPreset<P>::k;
    }
    t.NU = NU;
    std::vector<int> M((size_t)side * side, -1);
    std::vector<int> ux(NU), uy(NU);
    for (int q = 0; q < NU; ++q) {
        int c[3];
        host_lambda(f, q, L - U, c);
        ux[q] = c[0];
        uy[q] = c[1];
        M[(size_t)c[1] * side + c[0]] = q;
    }
    // the unit layout against the fractal's own lambda
    for (int q = 0; q < NU; ++q)
        for (int u = 0; u < NB; ++u) {
            int c[3];
            host_lambda(f, (int64_t)NB * q + u, L, c);
            if (c[0] != SIDE * ux[q] + lu_x<P, U>(u) || c[1] != SIDE * uy[q] + lu_y<P, U>(u)) return t;
        }
    std::vector<std::vector<int>> dir_bytes(8);   // per direction: the unit bytes the frame reads
    for (int e = 0; e < NE; ++e) {
        const int x = lu_ext_x<P, U>(e), y = lu_ext_y<P, U>(e);
        dir_bytes[lu_dir<P, U>(x, y)].push_back(lu_fbyte<P, U>(x, y));
    }
    std::map<std::pair<int, int>, int> slot_of;   // (tile-table slot, unit there) -> halo unit
    std::vector<std::pair<int, int>> slots;
    std::vector<std::vector<uint8_t>> bytes_read;
    std::vector<int> nb((size_t)NU * 8);
    for (int q = 0; q < NU; ++q)
        for (int d = 0; d < 8; ++d) {
            const int d9 = d < 4 ? d : d + 1;
            int nx = ux[q] + d9 % 3 - 1, ny = uy[q] + d9 / 3 - 1;
            const int tdx = nx < 0 ? -1 : (nx >= side ? 1 : 0), tdy = ny < 0 ? -1 : (ny >= side ? 1 : 0);
            nx = (nx + side) % side;
            ny = (ny + side) % side;
            const int gn = M[(size_t)ny * side + nx];
            int v = -2;   // -2: the zero unit
            if (gn >= 0 && !dir_bytes[d].empty()) {
                if (tdx == 0 && tdy == 0) v = gn;
                else {
                    const int t9 = (tdx + 1) + 3 * (tdy + 1);
                    const int tslot = t9 < 4 ? t9 : t9 - 1;
                    auto key = std::make_pair(tslot, gn);
                    auto it = slot_of.find(key);
                    if (it == slot_of.end()) {
                        it = slot_of.emplace(key, (int)slots.size()).first;
                        slots.push_back(key);
                        bytes_read.emplace_back(NB, 0);
                    }
                    for (int b : dir_bytes[d]) bytes_read[it->second][b] = 1;
                    v = -100 - it->second;
                }
            }
            nb[(size_t)q * 8 + d] = v;
        }
    t.H = (int)slots.size();
    const int64_t zero = NU + t.H;
    if ((int64_t)NB * zero + NB >= 65536) return t;
    t.words.assign((size_t)NU * 4, 0);
    for (int q = 0; q < NU; ++q)
        for (int d = 0; d < 8; ++d) {
            const int v = nb[(size_t)q * 8 + d];
            const uint32_t off = (v == -2) ? (uint32_t)(NB * zero)
                                 : (v <= -100 ? (uint32_t)(NB * (NU + (-100 - v))) : (uint32_t)(NB * v));
            t.words[(size_t)q * 4 + d / 2] |= off << (16 * (d % 2));
        }
    for (int hs = 0; hs < t.H; ++hs)
        for (int b = 0; b < NB; ++b) {
            if (!bytes_read[hs][b]) continue;
            t.ring.push_back((uint32_t)(NB * (NU + hs) + b) | ((uint32_t)slots[hs].first << 24));
            t.ring.push_back((uint32_t)(NB * slots[hs].second + b));
        }
    t.ok = true;
    return t;
}

struct Geometry {
    int mode, G, xoff, halo;
    int64_t B, Px, Py, planes;
    int64_t box_bytes, tab_entries, block;
    int64_t halo_bytes;   // stage bytes after the tile (ring-in-tile policies)
    int64_t data_bytes;   // if > 0: stage data bytes of a policy with padded units
};

static int64_t odd_words(int64_t px)
{
    px = (px + 3) / 4 * 4;
    if ((px / 4) % 2 == 0) px += 4;  // pitch/4 odd spreads block rows over banks
    return px;
}

static Geometry plan_geometry(const fractal *f, int L)
{
    Geometry g;
    g.B = ipow(f->s, L);
    g.G = group_levels(f);
    g.xoff = 0;
    g.block = 256;
    const bool grp = g.G > 0 && L >= g.G && ipow(f->k, g.G) <= kMaxGroup;
    g.halo = 0;
    g.halo_bytes = 0;
    g.data_bytes = 0;
    if (grp && is_triangle(f) && L >= 4 && ipow(f->k, L - 4) <= 256) {
        const TapTables t = tap_tables(f, L);
        if (t.ok) {
            g.mode = kModeTap;
            g.Px = g.Py = g.planes = 0;
            g.tab_entries = 0;   // the unit tables live in registers
            g.halo = t.H;
            g.halo_bytes = kTapHaloGap + 9 * (t.H + 1);
            g.block = std::max<int64_t>(64, ((int64_t)t.NQ + 31) / 32 * 32);
            g.box_bytes = 0;
            return g;
        }
    }
    const int rp = rows_preset_of(f);
    if (rp == kLidPreset && L >= kLidLevels && ipow(f->k, L - kLidLevels) <= 256) {
        const RowsTables t = lid_tables<kLidPreset, kLidLevels>(f, L);
        if (t.ok) {
            g.mode = kModeLid1;
            g.Px = g.Py = g.planes = 0;
            g.tab_entries = 0;   // the unit tables live in registers
            g.halo = t.H;
            g.halo_bytes = (int64_t)ipow(f->k, kLidLevels) * (t.H + 1);
            g.block = std::max<int64_t>(64, ((int64_t)t.NU + 31) / 32 * 32);
            g.box_bytes = 0;
            return g;
        }
    }
    if (rp >= 0 && L >= 2 && ipow(f->k, L - 2) <= 256) {
        const RowsTables t = rp == 0 ? rows_tables<0>(f, L) : rows_tables<1>(f, L);
        if (t.ok) {
            g.mode = rp == 0 ? kModeRows0 : kModeRows1;
            g.Px = g.Py = g.planes = 0;
            g.tab_entries = 0;   // the unit tables live in registers
            g.halo = t.H;
            g.halo_bytes = (int64_t)f->k * f->k * (t.H + 1);
            g.data_bytes = t.data_bytes;
            g.block = std::max<int64_t>(64, ((int64_t)t.NU + 31) / 32 * 32);
            g.box_bytes = 0;
            return g;
        }
    }
    if (bit3_ok(f, L)) {
        g.mode = kModeBit3;
        g.G = 0;
        g.Px = g.Py = g.planes = 0;
        g.tab_entries = 0;
        g.box_bytes = 0;
        return g;
    }
    if (f->dim == 3) {
        const int64_t Px = box3_pitch(g.B), vol = Px * (g.B + 2) * (g.B + 2);
        if (Px <= 64 && vol < 65536) {
            g.mode = kModeBox3;
            g.G = 0;
            g.Px = Px;
            g.Py = g.B + 2;
            g.planes = g.B + 2;
            g.tab_entries = 0;   // its 16-bit box offsets are read from global memory
            g.box_bytes = 2 * round16(vol + 16);            // the box, then the totals box
            return g;
        }
    }
    if (grp) {
        g.mode = (int)ipow(f->s, g.G);
        g.tab_entries = ipow(f->k, L - g.G);
        g.Py = g.B + 2;
        g.planes = 1;
        const int64_t units = (g.tab_entries + 3) / 4 + 1;
        if (g.mode == 4 && ipow(f->k, g.G) == kQuadKG && units <= 256) {
            g.mode = kModeQuad;
            g.xoff = 3;
            g.Px = odd_words(g.B + 8);
            g.block = std::max<int64_t>(64, (units + 31) / 32 * 32);  // one unit per thread
        } else {
            g.Px = odd_words(g.B + 4);
        }
    } else {
        g.mode = kModeCell;
        g.G = 0;
        g.Px = g.B + 2;
        g.Py = g.B + 2;
        g.planes = (f->dim == 3) ? g.B + 2 : 1;
        g.tab_entries = cells_below(f, L);
    }
    g.box_bytes = round16(g.Px * g.Py * g.planes + 16);
    return g;
}

// Shared memory, in order: `nstage` input stages (table row, front pad,
// tile bytes), their mbarriers, the box, the per-tile table, and the output
// stage (front pad, tile bytes).  The pads give the quad policy room for the
// partial units at both ends of a tile.
constexpr int kStagePad = 48;

struct Layout {
    int64_t nstage, stage_bytes, tile_bytes, off_bar, off_box, box_bytes, off_tab, off_out, total;
};

static Layout plan_layout(const fractal *f, int L)
{
    Layout y;
    Geometry g = plan_geometry(f, L);
    int64_t KL = cells_below(f, L);
    if (g.mode == kModeBit3) {
        // no stages: the shared tables, then each warp's box and buffer
        y = Layout();
        y.off_box = round16(4 * bit3_shared_words(f));
        y.total = y.off_box + (int64_t)kB3Warps * bit3_warp_bytes(f);
        return y;
    }
    y.nstage = (g.mode == kModeQuad || g.mode == kModeTap || g.mode == kModeRows0 || g.mode == kModeRows1 ||
                g.mode == kModeLid1 || g.mode == kModeBox3) ? 2 : nstages();
    if (f->stages_user >= 2) y.nstage = f->stages_user;
    // slack: 16-byte rounding of the bulk copy, whole-word reads and writes
    // past the tile's last cell; tap mode: halo and zero groups
    y.tile_bytes = round16((g.data_bytes > 0 ? g.data_bytes : KL + g.halo_bytes) + 64);
    y.stage_bytes = 4 * nbr_width(f->dim) + kStagePad + y.tile_bytes;
    int64_t off = y.nstage * y.stage_bytes;
    y.off_bar = off;
    off += 8 * y.nstage;
    off = round16(off);
    y.off_box = off;
    y.box_bytes = g.box_bytes;
    off += y.box_bytes;
    y.off_tab = off;
    off += round16(4 * g.tab_entries);
    y.off_out = off;
    // padded units and box3 store straight to memory
    // (warp w's bytes sit 16 w bytes further in, see one_barrier_loop)
    off += (g.data_bytes > 0 || g.mode == kModeBox3) ? 0 : kStagePad + y.tile_bytes + 16 * ((g.block + 31) / 32);
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
    while (best < f->r && cells_above(f, best) >= ((int64_t)1 << 31)) ++best;
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
        const int base = F.r - coarse_levels;   // the coarse levels sit above the tile's
        lambda64(F, (uint64_t)T, coarse_levels, c, base);
        int slot = 0;
        for (int q = 0; q < ndir; ++q) {
            int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (F.dim == 3) ? q / 9 - 1 : 0;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            int32_t qx = c[0] + dx, qy = c[1] + dy, qz = c[2] + dz;
            int64_t t = -1;
            if (qx >= 0 && qx < coarse_side && qy >= 0 && qy < coarse_side &&
                (F.dim == 2 || (qz >= 0 && qz < coarse_side)))
                t = nu_levels(F, qx, qy, F.dim == 3 ? qz : 0, coarse_levels, base);
            table[T * nbrw + slot++] = (int32_t)t;
        }
        for (; slot < nbrw; ++slot) table[T * nbrw + slot] = -1;
    }
}

template <int DIM, int MODE, bool MULTI>
__global__ void step_tma_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in,
                                uint8_t *__restrict__ out);

// The dynamic shared-memory limit is a property of the kernel function, shared
// by every handle: it is raised to the device's opt-in maximum (never set to
// one plan's size, which would break plans that need more).
template <int DIM, int MODE>
static int configure(StepPlan &p, int num_sms)
{
    int per_sm = 0, dev = 0, optin = 0;
    FR_CUDA(cudaGetDevice(&dev));
    FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (p.smem > optin) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    FR_CUDA(cudaFuncSetAttribute(step_tma_kernel<DIM, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaFuncSetAttribute(step_tma_kernel<DIM, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tma_kernel<DIM, MODE, false>, p.block, p.smem));
    if (per_sm < 1) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    p.per_sm = per_sm;
    p.grid = (int)std::min<int64_t>((int64_t)per_sm * num_sms, p.NT);
    return FR_OK;
}

template <bool MULTI, bool B5S45, int KW, bool IN_BITS, bool OUT_BITS>
__global__ void step_bit3_kernel(StepArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out);

// every instantiation of the bit3 kernel may use the opt-in shared memory
template <bool B5S45, int KW>
static int bit3_allow_smem(int optin)
{
    FR_CUDA(cudaFuncSetAttribute(step_bit3_kernel<false, B5S45, KW, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaFuncSetAttribute(step_bit3_kernel<false, B5S45, KW, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaFuncSetAttribute(step_bit3_kernel<false, B5S45, KW, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaFuncSetAttribute(step_bit3_kernel<false, B5S45, KW, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    if (!B5S45)
        FR_CUDA(cudaFuncSetAttribute(step_bit3_kernel<true, false, KW, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return FR_OK;
}

// shared memory of a states -> states generation: the tables and each warp's pointers
static int bit3_states_smem(const StepPlan &p) { return p.b3.off_warp + kB3Warps * kB3StatePtrBytes; }

// bit3 mode: eight tiles (warps) per block
static int configure_bit3(StepPlan &p, int num_sms)
{
    int per_sm = 0, dev = 0, optin = 0;
    FR_CUDA(cudaGetDevice(&dev));
    FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (p.smem > optin) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    int rc = bit3_allow_smem<false, 0>(optin);
    if (!rc) rc = bit3_allow_smem<true, 0>(optin);
    if (!rc) rc = bit3_allow_smem<false, 5>(optin);
    if (!rc) rc = bit3_allow_smem<true, 5>(optin);
    if (rc) return rc;
    FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_bit3_kernel<false, false, 0, false, false>, p.block, p.smem));
    {
        int per_sm_states = 0;
        FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_states, step_bit3_kernel<false, true, 5, true, true>,
                                                              p.block, bit3_states_smem(p)));
        p.b3.grid_states = (int)std::min<int64_t>((int64_t)std::max(per_sm_states, 1) * num_sms,
                                                  (p.NT + kB3Warps - 1) / kB3Warps);
    }
    if (per_sm < 1) {
        set_error(FR_EINVAL, "fractal_step: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    p.per_sm = per_sm;
    p.grid = (int)std::min<int64_t>((int64_t)per_sm * num_sms, (p.NT + kB3Warps - 1) / kB3Warps);
    return FR_OK;
}

// Selector nibble that yields a zero byte (sign of a byte whose msb is 0).
static constexpr uint32_t kZeroSel = 0x8;

int ensure_step_plan(fractal *f)
{
    // the plan depends only on the fractal and on these two settings (the
    // tables behind the automatic choice are too costly to rebuild per call)
    if (f->plan.pos && f->plan.built_levels == f->tile_levels_user && f->plan.built_stages == f->stages_user)
        return FR_OK;
    int L = choose_levels(f);
    free_step_plan(f->plan);
    int rc = ensure_status(f);
    if (rc) return rc;
    StepPlan p;
    p.L = L;
    p.KL = cells_below(f, L);
    p.NT = cells_above(f, L);
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
    p.xoff = geo.xoff;
    p.box_bytes = (int)y.box_bytes;
    p.stage_bytes = (int)y.stage_bytes;
    p.tile_bytes = (int)y.tile_bytes;
    p.off_bar = (int)y.off_bar;
    p.off_box = (int)y.off_box;
    p.off_pos = (int)y.off_tab;
    p.off_out = (int)y.off_out;
    p.smem = (int)y.total;
    p.nstage = (int)y.nstage;
    p.nbrw = nbr_width(f->dim);
    p.ntab = (int)geo.tab_entries;
    p.block = (int)geo.block;
    const int dim = f->dim;
    const int64_t W[3] = {geo.B + 2, geo.B + 2, dim == 3 ? geo.B + 2 : 1};  // padded extents
    auto offset_of = [&](const int b[3]) -> int64_t {
        return (b[0] + geo.xoff) + geo.Px * (b[1] + geo.Py * (int64_t)(dim == 3 ? b[2] : 0));
    };
    if (geo.Px * geo.Py * geo.planes >= (1 << 24)) {
        set_error(FR_EINVAL, "fractal_step: tile box too large");
        return FR_EINVAL;
    }

    std::vector<uint32_t> tab, ring;
    if (p.mode == kModeBit3) {
        tab = bit3_tables(f, p.b3);
        p.b3.off_warp = (int)y.off_box;
        p.b3.warp_bytes = bit3_warp_bytes(f);
        p.nstage = 0;
    } else if (p.mode == kModeTap) {
        const TapTables t = tap_tables(f, L);
        p.KG = 9;
        p.tapz = t.zero_off;
        p.nq = t.NQ;
        tab = t.words;
        ring = t.ring;
    } else if (p.mode == kModeLid1) {
        const RowsTables t = lid_tables<kLidPreset, kLidLevels>(f, L);
        p.KG = (int)ipow(f->k, kLidLevels);
        p.tapz = t.NU + t.H;
        p.nq = t.NU;
        tab = t.words;
        ring = t.ring;
    } else if (p.mode == kModeRows0 || p.mode == kModeRows1) {
        const RowsTables t = p.mode == kModeRows0 ? rows_tables<0>(f, L) : rows_tables<1>(f, L);
        p.KG = f->k * f->k;
        p.tapz = t.NU + t.H;
        p.nq = t.NU;
        tab = t.words;
        ring = t.halo.empty() ? t.ring : t.halo;
        p.nhalo = (int)t.halo.size() / 2;
        p.hbytes = t.hbytes;
        p.zoff = t.zoff;
    } else {
        // local lambda -> padded box offset; occupancy of the interior
        std::vector<uint32_t> pos(p.KL);
        std::vector<uint8_t> occ((size_t)(geo.Px * geo.Py * geo.planes + 16), 0);
        for (int64_t l = 0; l < p.KL; ++l) {
            int c[3];
            host_lambda(f, l, L, c);
            int b[3] = {c[0] + 1, c[1] + 1, c[2] + 1};
            int64_t o = offset_of(b);
            pos[l] = (uint32_t)o;
            occ[o] = 1;
        }
        if (p.mode == kModeBox3) {
            tab.assign((size_t)(p.KL + 3) / 4 * 2, 0u);
            for (int64_t l = 0; l < p.KL; ++l) tab[l / 2] |= pos[l] << (16 * (l % 2));
        } else if (p.mode != kModeCell) {
            // group g = cells [g k^G, (g+1) k^G); its block sits at s^G * (coarse
            // lambda of g over L - G levels); the window starts one cell up-left
            const int KG = (int)ipow(f->k, p.G), SG = (int)ipow(f->s, p.G);
            p.KG = KG;
            for (int q = 0; q < kMaxGroup; ++q) p.lid_of_q[q] = -1;
            for (int lid = 0; lid < KG; ++lid) {
                int c[3];
                host_lambda(f, lid, p.G, c);
                p.lid_of_q[c[1] * SG + c[0]] = (int8_t)lid;
                p.rel_of_lid[lid] = (int16_t)((c[1] + 1) * geo.Px + (c[0] + 1) + geo.xoff);
            }
            tab.resize(geo.tab_entries);
            for (int64_t g = 0; g < geo.tab_entries; ++g) {
                int c[3];
                host_lambda(f, g, L - p.G, c);
                tab[g] = (uint32_t)((int64_t)c[1] * SG * geo.Px + (int64_t)c[0] * SG);
            }
            if (p.mode == kModeQuad) {
                // block row j <- group cells: first permute over words 0,1 of the
                // group, then take cells 8..11 from word 2
                for (int j = 0; j < 4; ++j) {
                    uint32_t sa = 0, sb = 0;
                    for (int c = 0; c < 4; ++c) {
                        const int lid = p.lid_of_q[j * 4 + c];
                        const uint32_t na = (lid >= 0 && lid < 8) ? (uint32_t)lid : kZeroSel;
                        const uint32_t nb = (lid >= 8) ? (uint32_t)(4 + lid - 8) : (uint32_t)c;
                        sa |= na << (4 * c);
                        sb |= nb << (4 * c);
                    }
                    p.row_sel[2 * j] = sa;
                    p.row_sel[2 * j + 1] = sb;
                }
                // cell order word m <- block sums (16 bytes: row j, column c at 4j+c)
                for (int m = 0; m < 3; ++m) {
                    uint32_t sa = 0, sb = 0, sc = 0;
                    for (int i = 0; i < 4; ++i) {
                        const int lid = 4 * m + i;
                        uint32_t na = kZeroSel, nb = kZeroSel, nc = kZeroSel;
                        if (lid < KG) {
                            int c[3];
                            host_lambda(f, lid, p.G, c);
                            const int idx = 4 * c[1] + c[0];
                            if (idx < 8) { na = idx; nc = i; }
                            else { nb = idx - 8; nc = 4 + i; }
                        }
                        sa |= na << (4 * i);
                        sb |= nb << (4 * i);
                        sc |= nc << (4 * i);
                    }
                    p.pack_sel[3 * m] = sa;
                    p.pack_sel[3 * m + 1] = sb;
                    p.pack_sel[3 * m + 2] = sc;
                }
            }
        } else {
            tab = pos;
        }
        // halo ring: padded cells with some coordinate 0 or B+1 that are members
        // of their (wrapped) local box and touch an interior member
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

    }
    p.nring = p.nhalo ? 0 : (int)(ring.size() / 2);
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
    if (p.mode == kModeBit3) rc = configure_bit3(p, f->num_sms);
    else if (dim == 3) rc = p.mode == kModeBox3 ? configure<3, kModeBox3>(p, f->num_sms) : configure<3, kModeCell>(p, f->num_sms);
    else if (p.mode == kModeQuad) rc = configure<2, kModeQuad>(p, f->num_sms);
    else if (p.mode == kModeTap) rc = configure<2, kModeTap>(p, f->num_sms);
    else if (p.mode == kModeRows0) rc = configure<2, kModeRows0>(p, f->num_sms);
    else if (p.mode == kModeRows1) rc = configure<2, kModeRows1>(p, f->num_sms);
    else if (p.mode == kModeLid1) rc = configure<2, kModeLid1>(p, f->num_sms);
    else if (p.mode == kModeGroup4) rc = configure<2, kModeGroup4>(p, f->num_sms);
    else if (p.mode == kModeGroup3) rc = configure<2, kModeGroup3>(p, f->num_sms);
    else rc = configure<2, kModeCell>(p, f->num_sms);
    if (rc) {
        free_step_plan(p);
        return rc;
    }
    p.built_levels = f->tile_levels_user;
    p.built_stages = f->stages_user;
    f->plan = p;
    return FR_OK;
}

// ------------------------------------------------------------------ device

__device__ __forceinline__ uint32_t lds32(const uint8_t *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void sts32(uint8_t *p, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(p) = v;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// nonzero byte -> 1, zero byte -> 0
__device__ __forceinline__ uint32_t bytes_to_01(uint32_t v)
{
    return (((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v) >> 7 & 0x01010101u;
}

// Life-like rule on 4 cells at once: t = 3x3 sum including the cell (<= 9),
// alive = 0/1 bytes.  The look-up tables hold, in byte j, the outcome for a
// total of j in bit 0 and for a total of j + 8 in bit 7; prmt returns byte
// (t & 7), or its bit 7 replicated when t >= 8.
__device__ __forceinline__ uint32_t rule4(const uint32_t lut[4], uint32_t t, uint32_t alive)
{
    const uint32_t x = __umulhi(t, 1u << 28) + t;   // t | t >> 4 (totals < 16)
    const uint32_t sel = prmt(x, 0u, 0x3120u);   // nibble i = total of cell i
    const uint32_t rd = prmt(lut[0], lut[1], sel);
    const uint32_t rl = prmt(lut[2], lut[3], sel);
    // bit 0 of each byte: the live table's where the cell is alive (alive
    // bytes are 0 or 1), the dead table's elsewhere
    return ((rl & alive) | (rd & ~alive)) & 0x01010101u;
}

// The same on a fractal whose cells have at most 6 member neighbours: the
// nibble t + 8 alive (<= 14) picks bit 0 of byte t (dead cell, t
// neighbours) or, in prmt's sign mode, bit 7 of byte t (live cell, total t)
// of lut_sparse.
__device__ __forceinline__ uint32_t rule4_sparse(const uint32_t lut[2], uint32_t t, uint32_t alive)
{
    const uint32_t i = alive * 8u + t;
    const uint32_t x = __umulhi(i, 1u << 28) + i;   // i | i >> 4
    return prmt(lut[0], lut[1], prmt(x, 0u, 0x3120u)) & 0x01010101u;
}

// Window of the block of one group: rows r = 0..SG+1, bytes 0..SG+1 of the
// pair (lo, hi) are the window columns.  `ad0` is the byte address of the
// window's first column in row 0.  Three words per row cover any alignment.
template <int SG>
__device__ __forceinline__ void load_window(const uint8_t *box, uint32_t ad0, int Px, uint32_t *lo,
                                            uint32_t *hi)
{
#pragma unroll
    for (int r = 0; r < SG + 2; ++r) {
        const uint32_t ad = ad0 + r * Px;
        const uint32_t al = ad & ~3u;
        const uint32_t sh = (ad & 3u) * 8u;
        const uint32_t w0 = lds32(box + al), w1 = lds32(box + al + 4), w2 = lds32(box + al + 8);
        lo[r] = __funnelshift_r(w0, w1, sh);
        hi[r] = __funnelshift_r(w1, w2, sh);
    }
}

// New states of the cells of one group from its window (byte stores).
template <int SG>
__device__ __forceinline__ void group_from_window(const StepArgs &a, const Rule &rule,
                                                  const uint32_t *lo, const uint32_t *hi,
                                                  uint8_t *gout)
{
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
                gout[lid] = ((al ? rule.survive : rule.birth) >> cnt) & 1u;
            }
        }
    }
}

struct TileIO {
    const uint8_t *data;   // 16-byte aligned stage data; tile cell l at data[a_in + l]
    uint8_t *ostage;       // 16-byte aligned output stage; tile cell l at ostage[a_out + l]
    uint8_t *gout;         // the tile's first output cell in memory
    int a_in, a_out;
    Rule rule;             // the rule of the tile's instance
};

// ---- cell policy
template <int DIM>
struct CellPolicy {
    static constexpr int NDIR = (DIM == 3) ? 27 : 9;
    static constexpr bool kRingInTile = false;  // halo bytes go to the box
    struct Regs { int nb[NDIR - 1]; };
    __device__ static void init(const StepArgs &a, Regs &R)
    {
        const int PX = a.Px, PXY = a.Px * a.Py;
        int e = 0;
        for (int q = 0; q < NDIR; ++q) {
            int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = (DIM == 3) ? q / 9 - 1 : 0;
            if (dx == 0 && dy == 0 && dz == 0) continue;
            R.nb[e++] = dx + PX * dy + PXY * dz;
        }
    }
    __device__ static void scatter(const StepArgs &a, const TileIO &io, uint8_t *box,
                                   const uint32_t *tab, Regs &)
    {
        const uint8_t *tin = io.data + io.a_in;
        for (int64_t l = threadIdx.x; l < a.KL; l += blockDim.x) box[tab[l]] = tin[l] != 0;
    }
    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *box,
                                   const uint32_t *tab, Regs &R)
    {
        uint8_t *tout = io.ostage + io.a_out;
        for (int64_t l = threadIdx.x; l < a.KL; l += blockDim.x) {
            const int p = tab[l];
            int cnt = 0;
#pragma unroll
            for (int e = 0; e < NDIR - 1; ++e) cnt += box[p + R.nb[e]];
            const uint32_t mask = box[p] ? io.rule.survive : io.rule.birth;
            tout[l] = (mask >> cnt) & 1u;
        }
    }
};

// ---- group policy (one thread per group, byte stores)
template <int SG>
struct GroupPolicy {
    struct Regs {};
    static constexpr bool kRingInTile = false;  // halo bytes go to the box
    __device__ static void init(const StepArgs &, Regs &) {}
    __device__ static void scatter(const StepArgs &a, const TileIO &io, uint8_t *box,
                                   const uint32_t *tab, Regs &)
    {
        const uint8_t *tin = io.data + io.a_in;
        for (int g = threadIdx.x; g < a.ntab; g += blockDim.x) {
            const uint32_t base = tab[g];
            const uint8_t *src = tin + (int64_t)g * a.KG;
            for (int lid = 0; lid < a.KG; ++lid) box[base + a.rel_of_lid[lid]] = src[lid] != 0;
        }
    }
    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *box,
                                   const uint32_t *tab, Regs &)
    {
        uint8_t *tout = io.ostage + io.a_out;
        for (int g = threadIdx.x; g < a.ntab; g += blockDim.x) {
            uint32_t lo[SG + 2], hi[SG + 2];
            load_window<SG>(box, tab[g], a.Px, lo, hi);
            group_from_window<SG>(a, io.rule, lo, hi, tout + (int64_t)g * a.KG);
        }
    }
};

// ---- quad policy (s = 2, 9-cell groups, four groups per thread)
//
// Units of 4 consecutive groups start at group gs, the first group index
// (possibly negative) for which the output byte offset a_out + 9 gs is a
// multiple of 4, so every unit reads and writes whole words.  Groups of a
// unit that lie outside [0, NG) are computed from a valid block and their
// garbage lands in the padding before / after the tile in the stages; they
// never touch the box.
struct QuadPolicy {
    static constexpr int KG = kQuadKG;
    static constexpr bool kRingInTile = false;  // halo bytes go to the box
    struct Regs {
        uint32_t v[KG + 1];     // the unit's 36 input bytes as words (v[KG] = 0)
        uint32_t rw[4][4];      // block rows of the four groups
        int gq;                 // first group of the unit, or INT_MIN when idle
    };
    __device__ static void init(const StepArgs &, Regs &) {}

    __device__ static void scatter(const StepArgs &a, const TileIO &io, uint8_t *box,
                                   const uint32_t *tab, Regs &R)
    {
        int gs = 0;
        while ((io.a_out + KG * gs) & 3) ++gs;
        if (gs > 0) gs -= 4;
        const int ng = a.ntab;
        const int gq = gs + 4 * (int)threadIdx.x;
        R.gq = gq < ng ? gq : INT_MIN;
        if (R.gq == INT_MIN) return;
        const int off = io.a_in + KG * gq;          // may be negative: stage front padding
        const uint8_t *wp = io.data + (off & ~3);
        const uint32_t sh = (uint32_t)(off & 3) * 8u;
        uint32_t w[KG + 1];
#pragma unroll
        for (int i = 0; i <= KG; ++i) w[i] = lds32(wp + 4 * i);
        uint32_t any = 0;
#pragma unroll
        for (int i = 0; i < KG; ++i) {
            R.v[i] = __funnelshift_r(w[i], w[i + 1], sh);
            any |= R.v[i];
        }
        R.v[KG] = 0;
        if (any & 0xfefefefeu) {
#pragma unroll
            for (int i = 0; i < KG; ++i) R.v[i] = bytes_to_01(R.v[i]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b0 = KG * u;  // the group's 9 bytes start at byte 9u of v
            const uint32_t g0w = __funnelshift_r(R.v[b0 / 4], R.v[b0 / 4 + 1], (b0 % 4) * 8);
            const uint32_t g1w = __funnelshift_r(R.v[b0 / 4 + 1], R.v[b0 / 4 + 2], (b0 % 4) * 8);
            const uint32_t g2w = __funnelshift_r(R.v[b0 / 4 + 2], R.v[b0 / 4 + 3 <= KG ? b0 / 4 + 3 : KG], (b0 % 4) * 8);
            const int g = gq + u;
            const bool valid = g >= 0 && g < ng;
            const uint32_t base = tab[valid ? g : 0] + 4;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t x = prmt(g0w, g1w, a.row_sel[2 * j]);
                const uint32_t row = prmt(x, g2w, a.row_sel[2 * j + 1]);
                R.rw[u][j] = row;
                if (valid) sts32(box + base + (j + 1) * a.Px, row);
            }
        }
    }

    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *box,
                                   const uint32_t *tab, Regs &R)
    {
        if (R.gq == INT_MIN) return;
        const int ng = a.ntab;
        uint32_t T[KG + 1];
#pragma unroll
        for (int i = 0; i <= KG; ++i) T[i] = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int g = R.gq + u;
            const uint32_t base = tab[(g >= 0 && g < ng) ? g : 0];
            uint32_t lo[6], hi[6];
            // window rows 0 and 5 from the box; rows 1..4 reuse this group's
            // own block rows held in registers
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const uint8_t *rp = box + base + r * a.Px;
                const uint32_t w0 = lds32(rp);
                const uint32_t w1 = (r >= 1 && r <= 4) ? R.rw[u][r - 1] : lds32(rp + 4);
                const uint32_t w2 = lds32(rp + 8);
                lo[r] = __funnelshift_r(w0, w1, 24);
                hi[r] = __funnelshift_r(w1, w2, 24);
            }
            // vertical 3-row sums with shared pairs, then 3-column sums
            const uint32_t pl01 = lo[0] + lo[1], pl23 = lo[2] + lo[3], pl45 = lo[4] + lo[5];
            const uint32_t ph01 = hi[0] + hi[1], ph23 = hi[2] + hi[3], ph45 = hi[4] + hi[5];
            const uint32_t vl[4] = {pl01 + lo[2], lo[1] + pl23, pl23 + lo[4], lo[3] + pl45};
            const uint32_t vh[4] = {ph01 + hi[2], hi[1] + ph23, ph23 + hi[4], hi[3] + ph45};
            uint32_t S[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                S[j] = vl[j] + __funnelshift_r(vl[j], vh[j], 8) + __funnelshift_r(vl[j], vh[j], 16);
            // block sums -> the group's 9 cells in omega order, merged into
            // the unit's totals at byte 9u
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const uint32_t x = prmt(S[0], S[1], a.pack_sel[3 * m]);
                const uint32_t y = prmt(S[2], S[3], a.pack_sel[3 * m + 1]);
                const uint32_t tg = prmt(x, y, a.pack_sel[3 * m + 2]);
                const int b = KG * u + 4 * m;
                if (b / 4 <= KG) {
                    T[b / 4] |= tg << ((b % 4) * 8);
                    if ((b % 4) && b / 4 + 1 <= KG) T[b / 4 + 1] |= tg >> (32 - (b % 4) * 8);
                }
            }
        }
        uint8_t *op = io.ostage + io.a_out + KG * R.gq;   // word aligned; may start in the padding
#pragma unroll
        for (int i = 0; i < KG; ++i) sts32(op + 4 * i, rule4(io.rule.lut, T[i], R.v[i]));
    }
};

// ---- tap policy (the triangle; see kTap and kPosX): no box.  A thread
// owns one unit (9 groups, 81 cells).  Of the 8 taps of each group, those in
// a group of the same unit come from the thread's registers, those in a hole
// of the unit's block are 0, and the 14 external ones are read from the
// stage through the unit's 12 external group offsets, which are the same
// for every tile and stay in registers.  The totals of a group are summed
// in cell order: each of its three level-1 triangles (lids 0-2, 3-5, 6-8)
// gives its sum to its own three cells; the five edges between them (lids
// 1-3, 1-5, 2-6, 2-7, 5-7) and the taps add the rest.

// tap byte, 0 or 1, from its source (see tap_src)
template <int S>
__device__ __forceinline__ uint32_t tap_byte(const uint32_t *v, const uint32_t *x)
{
    if constexpr (S == kSrcZero) return 0u;
    else if constexpr (S >= kSrcExt) return x[S - kSrcExt];
    else return prmt(v[S >> 2], 0u, 0x4440u | (uint32_t)(S & 3));
}

// bytes P .. P+3 of a byte stream held in words
template <int P>
__device__ __forceinline__ uint32_t win(const uint32_t *v)
{
    if constexpr (P % 4 == 0) return v[P / 4];
    else return __funnelshift_r(v[P / 4], v[P / 4 + 1], 8 * (P % 4));
}

// Stream of a unit's totals: byte p = 9J + r of the unit comes from group
// J's word T0 (r < 4), T1 (r = 4..7) or byte 2 of T2 (r = 8), held in
// R[3J], R[3J + 1], R[3J + 2].  Each stream word is gathered with one prmt
// from two of them (two prmts where it touches three).
constexpr int st_reg(int p) { return 3 * (p / 9) + ((p % 9) < 4 ? 0 : ((p % 9) < 8 ? 1 : 2)); }
constexpr int st_byte(int p) { return (p % 9) < 4 ? p % 9 : ((p % 9) < 8 ? p % 9 - 4 : 2); }
// the k-th distinct register of stream word W (-1: none)
constexpr int st_word_reg(int W, int k)
{
    int regs[4] = {-1, -1, -1, -1}, n = 0;
    for (int i = 0; i < 4; ++i) {
        const int p = 4 * W + i;
        if (p >= kUnitCells) break;
        const int r = st_reg(p);
        bool seen = false;
        for (int j = 0; j < n; ++j) seen = seen || regs[j] == r;
        if (!seen) regs[n++] = r;
    }
    return regs[k];
}
// selector of byte i of word W: its byte in the pair (first reg, second
// reg) when `pair`, else in (prmt result, third reg); 4 (a zero) past the unit
constexpr uint32_t st_nibble(int W, int i, bool pair)
{
    const int p = 4 * W + i;
    if (p >= kUnitCells) return 4;
    const int r = st_reg(p), b = st_byte(p);
    if (pair) return (uint32_t)(r == st_word_reg(W, 1) ? 4 + b : (r == st_word_reg(W, 0) ? b : 4));
    return (uint32_t)(r == st_word_reg(W, 2) ? 4 + b : i);
}
constexpr uint32_t st_sel(int W, bool pair)
{
    return st_nibble(W, 0, pair) | st_nibble(W, 1, pair) << 4 | st_nibble(W, 2, pair) << 8 |
           st_nibble(W, 3, pair) << 12;
}

template <int W>
__device__ __forceinline__ uint32_t stream_word(const uint32_t *R)
{
    constexpr int r0 = st_word_reg(W, 0), r1 = st_word_reg(W, 1), r2 = st_word_reg(W, 2);
    constexpr uint32_t s1 = st_sel(W, true);
    if constexpr (r1 < 0 && s1 == 0x3210u) return R[r0];
    else if constexpr (r1 < 0) return prmt(R[r0], 0u, s1);
    else if constexpr (r2 < 0) return prmt(R[r0], R[r1], s1);
    else return prmt(prmt(R[r0], R[r1], s1), R[r2], st_sel(W, false));
}

template <int... W>
__device__ __forceinline__ void stream_words(const uint32_t *R, uint32_t *S, std::integer_sequence<int, W...>)
{
    ((S[W] = stream_word<W>(R)), ...);
}

// A 1 the compiler cannot see: additions written as a * kOne + b stay
// integer multiply-adds, which run on the FMA pipe, instead of becoming
// ALU additions (the ALU pipe, at half rate, is the tap kernel's busiest).
__constant__ uint32_t kOne = 1u;
__device__ __forceinline__ uint32_t mad_u32(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// totals (3x3 sums including the cell) of group J of a unit: lids 0..3 in
// R[3J], 4..7 in R[3J + 1], lid 8 in byte 2 of R[3J + 2]
template <int J>
__device__ __forceinline__ void unit_group(const uint32_t *v, const uint32_t *x, uint32_t *R)
{
    constexpr int b = 9 * J;
    const uint32_t A = win<b>(v), B = win<b + 4>(v);     // lids 0-3, 4-7 (bytes 0 or 1)
    const uint32_t P0 = A * 0x010101u;                   // byte 2: l0 + l1 + l2
    const uint32_t P1 = win<b + 3>(v) * 0x010101u;      // byte 2: l3 + l4 + l5
    const uint32_t P2 = win<b + 6>(v) * 0x010101u;      // byte 2: l6 + l7 + l8
    const uint32_t w4 = tap_byte<tap_src(J, 0)>(v, x), e0 = tap_byte<tap_src(J, 1)>(v, x);
    const uint32_t e2 = tap_byte<tap_src(J, 2)>(v, x), n8 = tap_byte<tap_src(J, 3)>(v, x);
    const uint32_t ne8 = tap_byte<tap_src(J, 4)>(v, x), s0 = tap_byte<tap_src(J, 5)>(v, x);
    const uint32_t s1 = tap_byte<tap_src(J, 6)>(v, x), sw4 = tap_byte<tap_src(J, 7)>(v, x);
    // lids 0..3: t0 + N8 + W4 | t0 + l3 + l5 + N8 | t0 + l6 + l7 + W4 | t1 + l1
    // (selector nibble 8: the sign of byte 0 replicated, i.e. 0)
    // (every addition a multiply-add: see kOne)
    const uint32_t one = kOne;
    R[3 * J] = mad_u32(n8, 0x00000101u,
                       mad_u32(w4, 0x00010001u,
                               mad_u32(mad_u32(prmt(P0, P1, 0x6222u), one, prmt(A, B, 0x1638u)), one,
                                       prmt(B, 0u, 0x4314u))));
    // lids 4..7: t1 + NE8 + E0 + E2 | t1 + l1 + l7 | t2 + l2 | t2 + l2 + l5
    R[3 * J + 1] = mad_u32(mad_u32(mad_u32(prmt(P1, P2, 0x6622u), one, prmt(A, 0u, 0x2214u)), one,
                                   prmt(B, 0u, 0x1434u)),
                           one, mad_u32(mad_u32(ne8, one, e0), one, e2));
    // lid 8 (byte 2): t2 + SW4 + S0 + S1
    R[3 * J + 2] = mad_u32(mad_u32(mad_u32(sw4, one, s0), one, s1), 0x10000u, P2);
}

// external tap cell C, 0 or 1, read from the stage
template <int C>
__device__ __forceinline__ uint32_t ext_tap(const uint8_t *tin, const uint32_t *e)
{
    constexpr int g = kXg[C], lid = kXlid[C];
    return min((uint32_t)tin[e[g] + lid], 1u);
}

template <int... C>
__device__ __forceinline__ void ext_taps(const uint8_t *tin, const uint32_t *e, uint32_t *x,
                                         std::integer_sequence<int, C...>)
{
    ((x[C] = ext_tap<C>(tin, e)), ...);
}

struct TapPolicy {
    static constexpr bool kRingInTile = true;   // halo bytes go after the tile's bytes
    static constexpr bool kPadded = false;      // the tile's bytes as one copy
    static constexpr bool kRingByAll = false;   // 8 halo cells per tile: one warp fills them
    static constexpr int NW = (kUnitCells + 3) / 4;   // 21 words per unit
    struct Regs {
        uint32_t e[kExtGroups];   // byte offsets 9 g of the unit's external groups
    };
    __device__ static void init(const StepArgs &a, Regs &R)
    {
        const int q = threadIdx.x;
#pragma unroll
        for (int k = 0; k < kExtGroups / 2; ++k) {
            const uint32_t w = (q < a.nq) ? __ldg(a.tab + (kExtGroups / 2) * q + k) : 0u;
            R.e[2 * k] = w & 0xffffu;
            R.e[2 * k + 1] = w >> 16;
        }
    }
    // the all-zero group, after the halo groups (whatever was there before),
    // written by lanes 0..8 of the warp that fills the stage; `tin` is the
    // tile's first cell in the stage
    __device__ static void fill(const StepArgs &a, uint8_t *tin, int lane)
    {
        if (lane < 9) tin[a.tapz + lane] = 0;
    }
    // the tile bytes warp w writes: those of units 32w .. 32w + 31
    __device__ static void warp_bytes(const StepArgs &a, int w, int *b0, int *b1)
    {
        *b0 = kUnitCells * min(32 * w, a.nq);
        *b1 = kUnitCells * min(32 * w + 32, a.nq);
    }
    __device__ static void scatter(const StepArgs &, const TileIO &, uint8_t *, const uint32_t *, Regs &) {}

    __device__ static void compute(const StepArgs &a, const TileIO &io, const uint8_t *, const uint32_t *,
                                   Regs &R)
    {
        const int q = threadIdx.x;
        if (q >= a.nq) return;
        const uint8_t *tin = io.data + io.a_in;
        const int off = io.a_in + kUnitCells * q;
        const uint8_t *wp = io.data + (off & ~3);
        const uint32_t sh = (uint32_t)(off & 3) * 8u;
        // the unit's 81 cells (bytes 81..83 of v belong to whoever follows)
        uint32_t v[NW];
        uint32_t x[kExtCells];
        {
            uint32_t w[NW + 1];
#pragma unroll
            for (int i = 0; i <= NW; ++i) w[i] = lds32(wp + 4 * i);
            uint32_t any = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                v[i] = __funnelshift_r(w[i], w[i + 1], sh);
                any |= (i == NW - 1) ? (v[i] & 0xffu) : v[i];
            }
            if (any & 0xfefefefeu) {
#pragma unroll
                for (int i = 0; i < NW; ++i) v[i] = bytes_to_01(v[i]);
            }
            ext_taps(tin, R.e, x, std::make_integer_sequence<int, kExtCells>());
        }
        uint32_t T[3 * kUnitGroups];
        unit_group<0>(v, x, T);
        unit_group<1>(v, x, T);
        unit_group<2>(v, x, T);
        unit_group<3>(v, x, T);
        unit_group<4>(v, x, T);
        unit_group<5>(v, x, T);
        unit_group<6>(v, x, T);
        unit_group<7>(v, x, T);
        unit_group<8>(v, x, T);
        uint32_t o[NW];
        stream_words(T, o, std::make_integer_sequence<int, NW>());
#pragma unroll
        for (int i = 0; i < NW; ++i) o[i] = rule4_sparse(io.rule.lut_sparse, o[i], v[i]);
        // store bytes 0..80 of o at ob: word i of the aligned run from ob - m
        // holds stream bytes 4i - m .. 4i - m + 3; words 1..19 are the
        // unit's own, words 0 and 20 are shared with the neighbouring units
        // unless m = 0 (word 0) or m = 3 (word 20) and are written byte by byte
        uint8_t *ob = io.ostage + io.a_out + kUnitCells * q;
        const uint32_t m = (uint32_t)(io.a_out + kUnitCells * q) & 3u;
        uint8_t *base = ob - m;
        const uint32_t sl = 8u * m;
#pragma unroll
        for (int i = 1; i < NW - 1; ++i) sts32(base + 4 * i, __funnelshift_l(o[i - 1], o[i], sl));
        const uint32_t w0 = o[0] << sl, w20 = __funnelshift_l(o[NW - 2], o[NW - 1], sl);
        if (m == 0) sts32(base, w0);
        else {
#pragma unroll
            for (int j = 1; j < 4; ++j)
                if ((uint32_t)j >= m) base[j] = (uint8_t)(w0 >> (8 * j));
        }
        if (m == 3) sts32(base + 4 * (NW - 1), w20);
        else {
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if ((uint32_t)j <= m) base[4 * (NW - 1) + j] = (uint8_t)(w20 >> (8 * j));
        }
    }
};

}  // namespace fr
#include "rows.cuh"
#include "lid.cuh"
#include "box3.cuh"
#include "temporal.cuh"
namespace fr {

template <int DIM, int MODE>
struct PolicyOf;
template <int DIM>
struct PolicyOf<DIM, kModeCell> { using type = CellPolicy<DIM>; };
template <>
struct PolicyOf<2, kModeGroup3> { using type = GroupPolicy<3>; };
template <>
struct PolicyOf<2, kModeGroup4> { using type = GroupPolicy<4>; };
template <>
struct PolicyOf<2, kModeQuad> { using type = QuadPolicy; };
template <>
struct PolicyOf<2, kModeTap> { using type = TapPolicy; };
template <>
struct PolicyOf<2, kModeRows0> { using type = RowsPolicy<0>; };
template <>
struct PolicyOf<2, kModeRows1> { using type = RowsPolicy<1>; };
template <>
struct PolicyOf<2, kModeLid1> { using type = LidPolicy<kLidPreset, kLidLevels>; };
template <>
struct PolicyOf<3, kModeBox3> { using type = Box3Policy; };

// A tile of the launch resolved to its instance's buffers, table and rule.
struct TileRef {
    const uint8_t *in;
    uint8_t *out;
    const int32_t *nbr;
    int64_t cells;
    int64_t T;            // tile index within the instance
};

template <bool MULTI>
__device__ __forceinline__ TileRef resolve(const StepArgs &a, const uint8_t *in, uint8_t *out,
                                           int64_t Tg)
{
    TileRef t;
    if (!MULTI) {
        t.in = in;
        t.out = out;
        t.nbr = a.nbr;
        t.cells = a.cells;
        t.T = a.tile0 + Tg;
    } else {
        const InstDesc *d = a.insts + __ldg(a.tile_inst + Tg);
        if (a.gen & 1) {
            t.in = (a.gen == 1) ? d->first : d->even_dst;
            t.out = d->odd_dst;
        } else {
            t.in = d->odd_dst;
            t.out = d->even_dst;
        }
        t.nbr = d->nbr;
        t.cells = d->cells;
        t.T = Tg - d->tile0;
    }
    return t;
}

template <bool MULTI>
__device__ __forceinline__ void tile_rule(const StepArgs &a, int64_t Tg, Rule &r)
{
    if (!MULTI) r = a.rule;
    else r = a.insts[__ldg(a.tile_inst + Tg)].rule;
}

}  // namespace fr
#include "bit3.cuh"
namespace fr {

// Issue the bulk loads of a tile into one stage: its table row and the
// 16-byte-aligned part of its bytes that lies inside the instance's buffer.
__device__ __forceinline__ void issue_tile(const StepArgs &a, const TileRef &t, uint8_t *stage,
                                           uint64_t *bar)
{
    const uintptr_t start = (uintptr_t)(t.in + t.T * a.KL);
    const uintptr_t end = start + (uintptr_t)a.KL;
    const uintptr_t lo = start & ~(uintptr_t)15;
    const uintptr_t in_lo = ((uintptr_t)t.in + 15) & ~(uintptr_t)15;
    const uintptr_t in_hi = ((uintptr_t)t.in + (uintptr_t)t.cells) & ~(uintptr_t)15;
    uintptr_t b0 = lo > in_lo ? lo : in_lo;
    uintptr_t b1 = ((end + 15) & ~(uintptr_t)15);
    if (b1 > in_hi) b1 = in_hi;
    const uint32_t row_bytes = 4u * (uint32_t)a.nbrw;
    const uint32_t data_bytes = b1 > b0 ? (uint32_t)(b1 - b0) : 0u;
    mbar_arrive_expect_tx(bar, row_bytes + data_bytes + a.extra_tx);
    bulk_g2s(stage, t.nbr + t.T * a.nbrw, row_bytes, bar);
    if (data_bytes) bulk_g2s(stage + row_bytes + kStagePad + (b0 - lo), (const void *)b0, data_bytes, bar);
}

// After a failed wait: wait (bounded, with the default limit) for the bulk
// loads still in flight into this block's stages, those of the block's tiles
// j0 .. j1 (its iteration numbers), so that no copy lands after the block has
// exited.  Bytes a test armed beyond the copies (extra_tx) are counted as
// arrived first, so each stage completes exactly when its real copies have.
__device__ __forceinline__ void drain_loads(const StepArgs &a, uint64_t *bars, int64_t j0, int64_t j1)
{
    if (threadIdx.x != 0) return;
    for (int64_t j = j0; j <= j1; ++j) {
        if (blockIdx.x + j * (int64_t)gridDim.x >= a.NT) break;
        if (a.extra_tx) mbar_complete_tx(&bars[j % a.nstage], a.extra_tx);
        mbar_wait_bounded(&bars[j % a.nstage], (uint32_t)((j / a.nstage) & 1));
    }
}

// Input and output stage geometry of one tile.
__device__ __forceinline__ TileIO tile_io(const StepArgs &a, const TileRef &t, uint8_t *stage, uint8_t *ostage)
{
    const uintptr_t start = (uintptr_t)(t.in + t.T * a.KL);
    const uintptr_t ostart = (uintptr_t)(t.out + t.T * a.KL);
    TileIO io;
    io.data = stage + 4 * a.nbrw + kStagePad;   // data[j] <-> address (start & ~15) + j
    io.ostage = ostage;
    io.a_in = (int)(start & 15);
    io.a_out = (int)(ostart & 15);
    io.gout = t.out + t.T * a.KL;
    return io;
}

// Zero bytes in device memory, 16-byte aligned: the source of the halo
// runs whose tile is absent (padded-unit policies, runs of <= kRunMax units).
__device__ __align__(16) uint8_t g_zero_run[64 * kRunMax];

// A thread's first run of halo units (padded-unit policies): its two table
// words and, when `pre`, the table entry of its neighbouring tile for the
// tile about to be issued, loaded ahead of time.
struct HaloRun {
    uint32_t w0, w1;
    int32_t tn;
    bool pre;
};
// The first halo run of thread tid: the last warp's threads take the runs
// first, so that warp 0 (which arms the stage and copies the unit groups)
// and the last warp share the issue work.
__device__ __forceinline__ int first_halo_run(int tid, int nth)
{
    return tid + 32 < nth ? tid + 32 : tid + 32 - nth;
}

// Issue the copies of a tile into a stage: one bulk copy of the tile's bytes
// by lane 0 of warp 0, or (policies with padded units, called by every
// warp) one per group of units into their slots and one per run of halo
// units (`hr`: this thread's first run, or null).
template <bool MULTI, class Pol>
__device__ __forceinline__ void issue_stage(const StepArgs &a, const TileRef &t, uint8_t *stage, uint64_t *bar,
                                            const HaloRun *hr = nullptr)
{
    const int lane = threadIdx.x & 31;
    if constexpr (!Pol::kPadded) {
        if (lane == 0) {
            fence_proxy_async_smem();
            issue_tile(a, t, stage, bar);
        }
    } else {
        // padded units, by every warp of the block: lane l < 16 of warp w
        // copies unit groups 16 w + l, 16 (w + warps) + l, ... (the units
        // past the last whole group one by one, by threads 32 on), each
        // thread its halo runs (first_halo_run on, absent ones from zeros
        // in device memory), and thread 0 arms the stage with the byte count
        // of them all; a buffer that is not 16-byte aligned is copied with
        // plain loads and stores by warp 0 before it arms
        static_assert(Pol::NB * kRunMax <= (int)sizeof(g_zero_run), "zero run");
        constexpr int NB = Pol::NB;
        const int tid = threadIdx.x, warp = tid >> 5;
        const uint32_t row_bytes = 4u * (uint32_t)a.nbrw;
        uint8_t *data = stage + row_bytes + kStagePad;
        const uint8_t *src = t.in + t.T * a.KL;
        const int32_t *nrow = t.nbr + t.T * a.nbrw;
        const bool al = ((uintptr_t)src & 15) == 0;
        fence_proxy_async_smem();
        if (!al) {
            if (warp == 0) {
                for (int h = lane; h < a.nhalo; h += 32) {
                    const uint32_t w0 = __ldg(a.ring + 2 * h), w1 = __ldg(a.ring + 2 * h + 1);
                    const int32_t tn = __ldg(nrow + (w0 >> 24));
                    uint8_t *dst = data + (w1 >> 8);
                    const uint8_t *hs = tn < 0 ? g_zero_run : t.in + (int64_t)tn * a.KL + (int64_t)NB * (w0 & 0xffffffu);
                    for (int b = 0; b < NB * (int)(w1 & 0xffu); ++b) dst[b] = hs[b];
                }
                for (int u = lane; u < a.nq; u += 32)
                    for (int b = 0; b < NB; ++b) data[Pol::slot(u) + b] = src[NB * u + b];
                __threadfence_block();
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive_expect_tx(bar, row_bytes + a.extra_tx);
                    bulk_g2s(stage, nrow, row_bytes, bar);
                }
            }
            return;
        }
        if (tid == 0) {
            mbar_arrive_expect_tx(bar, row_bytes + (uint32_t)(a.nq * NB + a.hbytes) + a.extra_tx);
            bulk_g2s(stage, nrow, row_bytes, bar);
        }
        constexpr int G = Pol::kGroup;
        const int ng = a.nq / G, rem = a.nq - G * ng;
        for (int p = 16 * warp + lane; lane < 16 && p < ng; p += 16 * (int)(blockDim.x >> 5))
            bulk_g2s(data + Pol::slot(G * p), src + G * NB * p, G * NB, bar);
        if (tid >= 32 && tid < 32 + rem) {
            const int u = G * ng + tid - 32;
            bulk_g2s(data + Pol::slot(u), src + NB * u, NB, bar);
        }
        const int h0 = first_halo_run(tid, blockDim.x);
        for (int h = h0; h < a.nhalo; h += blockDim.x) {
            uint32_t w0, w1;
            int32_t tn;
            if (h == h0 && hr) {
                w0 = hr->w0;
                w1 = hr->w1;
                tn = hr->pre ? hr->tn : __ldg(nrow + (w0 >> 24));
            } else {
                w0 = __ldg(a.ring + 2 * h);
                w1 = __ldg(a.ring + 2 * h + 1);
                tn = __ldg(nrow + (w0 >> 24));
            }
            const uint8_t *hs = tn < 0 ? g_zero_run : t.in + (int64_t)tn * a.KL + (int64_t)NB * (w0 & 0xffffffu);
            bulk_g2s(data + (w1 >> 8), hs, (uint32_t)NB * (w1 & 0xffu), bar);
        }
    }
}

// Complete a landed stage for the compute of a ring-in-tile policy.  The
// last warp writes the tile bytes the bulk copy could not cover (within 16
// bytes of an unaligned end of the instance's buffer) and the policy's own
// bytes; every thread writes its share of the halo cells, entries tid + k *
// blockDim for k < kRingRegs from `rv` when they were prefetched.
template <bool MULTI, class Pol>
__device__ __forceinline__ void fill_stage(const StepArgs &a, const TileRef &t, uint8_t *stage, bool filler,
                                           const uint32_t *rv, bool pref)
{
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
    const int32_t *nrow = reinterpret_cast<const int32_t *>(stage);
    const uintptr_t start = (uintptr_t)(t.in + t.T * a.KL);
    uint8_t *tin = stage + 4 * a.nbrw + kStagePad + (Pol::kPadded ? 0 : (int)(start & 15));
    if constexpr (Pol::kPadded) {
        // the tile's units and halo units arrive by copies (issue_stage)
    } else if (filler) {
        // the bulk copy covered [cf, ct)
        const uintptr_t end = start + (uintptr_t)a.KL;
        const uintptr_t in_lo = ((uintptr_t)t.in + 15) & ~(uintptr_t)15;
        const uintptr_t in_hi = ((uintptr_t)t.in + (uintptr_t)t.cells) & ~(uintptr_t)15;
        const uintptr_t cf = start > in_lo ? start : in_lo, ct = end < in_hi ? end : in_hi;
        if (cf >= ct) {
            for (int64_t l = lane; l < a.KL; l += 32) tin[l] = ((const uint8_t *)start)[l];
        } else {
            if ((uintptr_t)lane < cf - start) tin[lane] = ((const uint8_t *)start)[lane];
            if ((uintptr_t)lane < end - ct) tin[ct - start + lane] = ((const uint8_t *)ct)[lane];
        }
        Pol::fill(a, tin, lane);
    }
    if constexpr (!Pol::kRingByAll) {
        // a short ring: the filling warp alone, entry `lane` prefetched
        for (int e = filler ? lane : a.nring; e < a.nring; e += 32) {
            const uint32_t w0 = __ldg(a.ring + 2 * e);
            uint32_t v = rv[0];
            if (!pref || e != lane) {
                const int32_t tn = nrow[w0 >> 24];
                v = (tn >= 0) ? t.in[(int64_t)tn * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
            }
            tin[w0 & 0xffffff] = v != 0;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRingRegs; ++k) {
            const int e = tid + k * nth;
            if (e < a.nring) {
                const uint32_t w0 = __ldg(a.ring + 2 * e);
                uint32_t v = rv[k];
                if (!pref) {
                    const int32_t tn = nrow[w0 >> 24];
                    v = (tn >= 0) ? t.in[(int64_t)tn * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
                }
                tin[w0 & 0xffffff] = v != 0;
            }
        }
        for (int e = tid + kRingRegs * nth; e < a.nring; e += nth) {
            const uint32_t w0 = __ldg(a.ring + 2 * e);
            const int32_t tn = nrow[w0 >> 24];
            const uint32_t v = (tn >= 0) ? t.in[(int64_t)tn * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
            tin[w0 & 0xffffff] = v != 0;
        }
    }
}

// Tile loop of the policies that compute from the input stage itself, with
// one block barrier per tile.  After computing tile i, each warp stores its
// own bytes of the output stage (a bulk copy of their 16-byte aligned part,
// plain stores for the ends) and waits for that copy to have read them
// before it writes the output stage again.  Tile byte j of warp w sits at
// 16 w + (the tile's output address mod 16) + j, so that a warp's bytes of
// one tile never overlap another warp's bytes of another tile; every thread waits for tile
// i+1's stage and fills its share of it, and the barrier that follows both
// closes tile i and opens tile i+1.  After it, thread 0 refills tile i's
// input stage.
template <bool MULTI, class Pol>
__device__ __forceinline__ void one_barrier_loop(const StepArgs &a, const uint8_t *in, uint8_t *out,
                                                 uint8_t *smem, uint64_t *bars, const uint32_t *tab,
                                                 typename Pol::Regs &R)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool filler = warp == (int)(blockDim.x >> 5) - 1;
    const int64_t G = gridDim.x;
    uint8_t *ostage = smem + a.off_out + kStagePad + 16 * warp;   // this warp's view
    int wb0, wb1;   // this warp's bytes of a tile
    Pol::warp_bytes(a, warp, &wb0, &wb1);
    int64_t Tg = blockIdx.x;
    if (Tg >= a.NT) return;
    uint32_t rv[kRingRegs];   // prefetched halo values of the next tile
#pragma unroll
    for (int k = 0; k < kRingRegs; ++k) rv[k] = 0;
    HaloRun hr{0u, 0u, 0, false};   // padded units: this thread's first halo run
    const bool has_run = Pol::kPadded && first_halo_run(tid, blockDim.x) < a.nhalo;
    if (has_run) {
        hr.w0 = __ldg(a.ring + 2 * first_halo_run(tid, blockDim.x));
        hr.w1 = __ldg(a.ring + 2 * first_halo_run(tid, blockDim.x) + 1);
    }
    TileRef t = resolve<MULTI>(a, in, out, Tg);
    bool ok = mbar_wait_bounded(&bars[0], 0, a.wait_limit);
    if (ok) fill_stage<MULTI, Pol>(a, t, smem, filler, rv, false);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(a.status, FR_ETIMEOUT);
        drain_loads(a, bars, 0, a.nstage - 1);
        return;
    }
    int s = 0;   // stage of tile i (the block's i-th), the next tile's stage and parity
    int sn = (a.nstage > 1) ? 1 : 0;
    uint32_t pn = (sn == 0) ? 1u : 0u;
    for (int64_t i = 0;; ++i) {
        uint8_t *stage = smem + s * a.stage_bytes;
        const int64_t Tn = Tg + G;
        const bool has_next = Tn < a.NT;
        uint8_t *next_stage = smem + sn * a.stage_bytes;
        TileRef tn = t;
        if (has_next) tn = resolve<MULTI>(a, in, out, Tn);
        // the next tile's halo values, when its stage has landed already
        // (never waited for here): the loads stay in flight during the compute
        bool pref = false;
        if constexpr (!Pol::kRingByAll) {
            if (filler && has_next && lane < a.nring && mbar_test(&bars[sn], pn)) {
                const uint32_t w0 = __ldg(a.ring + 2 * lane);
                const int32_t tnb = reinterpret_cast<const int32_t *>(next_stage)[w0 >> 24];
                rv[0] = (tnb >= 0) ? tn.in[(int64_t)tnb * a.KL + __ldg(a.ring + 2 * lane + 1)] : 0u;
                pref = true;
            }
        } else if (has_next && tid < a.nring && mbar_test(&bars[sn], pn)) {
            const int32_t *nrow_n = reinterpret_cast<const int32_t *>(next_stage);
#pragma unroll
            for (int k = 0; k < kRingRegs; ++k) {
                const int e = tid + k * (int)blockDim.x;
                if (e < a.nring) {
                    const uint32_t w0 = __ldg(a.ring + 2 * e);
                    const int32_t tnb = nrow_n[w0 >> 24];
                    rv[k] = (tnb >= 0) ? tn.in[(int64_t)tnb * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
                }
            }
            pref = true;
        }
        if constexpr (Pol::kPadded) {
            // the neighbouring tile of this thread's halo run for the tile
            // this stage is refilled with, loaded before the compute so that
            // the refill does not wait for it
            const int64_t Tr = Tg + a.nstage * G;
            if (has_run && Tr < a.NT) {
                const TileRef r = resolve<MULTI>(a, in, out, Tr);
                hr.tn = __ldg(r.nbr + r.T * a.nbrw + (hr.w0 >> 24));
                hr.pre = true;
            }
        }
        TileIO io = tile_io(a, t, stage, ostage);
        tile_rule<MULTI>(a, Tg, io.rule);
        if constexpr (Pol::kPadded) {
            // padded units: each thread writes its unit straight to memory
            Pol::compute(a, io, nullptr, tab, R);
        } else {
        if (lane == 0) bulk_wait_read_all();   // this warp's previous store has read its bytes
        __syncwarp();
        Pol::compute(a, io, nullptr, tab, R);
        fence_proxy_async_smem();             // this thread's writes, before the bulk copy reads them
        __syncwarp();
        if (wb1 > wb0) {
            // ostage[al + j] holds tile byte j; the warp's bytes [wb0, wb1)
            // are a bulk copy between their first and last 16-byte
            // boundaries in memory and plain stores around them
            uint8_t *ob = t.out + t.T * a.KL;
            const int al = io.a_out;
            const int head = (16 - ((al + wb0) & 15)) & 15, tail = (al + wb1) & 15;
            const int n = wb1 - wb0;
            if (n > head + tail) {
                if (lane == 0) {
                    bulk_s2g(ob + wb0 + head, ostage + al + wb0 + head, (uint32_t)(n - head - tail));
                    bulk_commit();
                }
                if (lane < head) ob[wb0 + lane] = ostage[al + wb0 + lane];
                else if (lane >= 16 && lane < 16 + tail) ob[wb1 - tail + lane - 16] = ostage[al + wb1 - tail + lane - 16];
            } else {
                for (int j = wb0 + lane; j < wb1; j += 32) ob[j] = ostage[al + j];
            }
        }
        }
        ok = true;
        if (has_next) {
            ok = mbar_wait_bounded(&bars[sn], pn, a.wait_limit);
            if (ok) fill_stage<MULTI, Pol>(a, tn, next_stage, filler, rv, pref);
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.status, FR_ETIMEOUT);
            drain_loads(a, bars, i + 1, i + a.nstage - 1);
            break;
        }
        if (Pol::kPadded || warp == 0) {
            const int64_t Tr = Tg + a.nstage * G;
            if (Tr < a.NT) issue_stage<MULTI, Pol>(a, resolve<MULTI>(a, in, out, Tr), stage, &bars[s], &hr);
        }
        if (!has_next) break;
        Tg = Tn;
        t = tn;
        s = sn;
        sn = (sn + 1 == a.nstage) ? 0 : sn + 1;
        if (sn == 0) pn ^= 1u;
    }
    if (!Pol::kPadded && lane == 0) bulk_wait_all();
}

// Whether a box policy writes its results straight to memory (io.gout)
// rather than to the output stage: the policy's kDirectStore, else false.
template <class Pol, class = void>
struct DirectStore {
    static constexpr bool value = false;
};
template <class Pol>
struct DirectStore<Pol, std::void_t<decltype(Pol::kDirectStore)>> {
    static constexpr bool value = Pol::kDirectStore;
};

// Tile loop of the policies that compute from the box: wait for the tile's
// stage; scatter its cells and halo into the box (halo values prefetched
// into registers during the previous tile when its stage had landed);
// barrier; refill the stage with the tile nstage iterations ahead; compute
// into the output stage; barrier; bulk-store the output stage.
template <bool MULTI, class Pol>
__device__ __forceinline__ void staged_loop(const StepArgs &a, const uint8_t *in, uint8_t *out, uint8_t *smem,
                                            uint64_t *bars, uint8_t *box, const uint32_t *tab,
                                            typename Pol::Regs &R)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t G = gridDim.x;
    const uint32_t row_bytes = 4u * (uint32_t)a.nbrw;
    uint8_t *ostage = smem + a.off_out + kStagePad;
    uint32_t rv[kRingRegs];   // prefetched halo values of the current tile
#pragma unroll
    for (int k = 0; k < kRingRegs; ++k) rv[k] = 0;
    bool pref = false;

    int64_t i = 0;
    int s = 0;             // stage of the block's i-th tile and the parity of its wait
    uint32_t parity = 0;
    for (int64_t Tg = blockIdx.x; Tg < a.NT;
         Tg += G, ++i, s = (s + 1 == a.nstage) ? 0 : s + 1, parity ^= (s == 0) ? 1u : 0u) {
        uint8_t *stage = smem + s * a.stage_bytes;
        const int32_t *nrow = reinterpret_cast<const int32_t *>(stage);
        const bool ok = mbar_wait_bounded(&bars[s], parity, a.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.status, FR_ETIMEOUT);
            drain_loads(a, bars, i, i + a.nstage - 1);
            break;
        }
        const TileRef t = resolve<MULTI>(a, in, out, Tg);
        const uintptr_t in_lo = ((uintptr_t)t.in + 15) & ~(uintptr_t)15;
        const uintptr_t in_hi = ((uintptr_t)t.in + (uintptr_t)t.cells) & ~(uintptr_t)15;
        const uintptr_t start = (uintptr_t)(t.in + t.T * a.KL);
        const uintptr_t end = start + (uintptr_t)a.KL;
        const uintptr_t lo = start & ~(uintptr_t)15;
        uint8_t *data = stage + row_bytes + kStagePad;   // data[j] <-> address lo + j
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
        const uintptr_t ostart = (uintptr_t)(t.out + t.T * a.KL);
        const uintptr_t oend = ostart + (uintptr_t)a.KL;
        const uintptr_t olo = ostart & ~(uintptr_t)15;
        TileIO io;
        io.data = data;
        io.ostage = ostage;
        io.a_in = (int)(start - lo);
        io.a_out = (int)(ostart - olo);
        io.gout = (uint8_t *)ostart;
        tile_rule<MULTI>(a, Tg, io.rule);

        Pol::scatter(a, io, box, tab, R);
        uint8_t *rdst = Pol::kRingInTile ? data + io.a_in : box;
        // halo cells: the first kRingRegs per thread were prefetched during the
        // previous tile (when `pref`), the rest are loaded now
#pragma unroll
        for (int k = 0; k < kRingRegs; ++k) {
            const int e = tid + k * nth;
            if (e < a.nring) {
                const uint32_t w0 = __ldg(a.ring + 2 * e);
                uint32_t v = rv[k];
                if (!pref) {
                    const int32_t tn = nrow[w0 >> 24];
                    v = (tn >= 0) ? t.in[(int64_t)tn * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
                }
                rdst[w0 & 0xffffff] = v != 0;
            }
        }
        for (int e = tid + kRingRegs * nth; e < a.nring; e += nth) {
            const uint32_t w0 = __ldg(a.ring + 2 * e), lw = __ldg(a.ring + 2 * e + 1);
            const int32_t tn = nrow[w0 >> 24];
            uint8_t v = 0;
            if (tn >= 0) v = t.in[(int64_t)tn * a.KL + lw] != 0;
            rdst[w0 & 0xffffff] = v;
        }
        // prefetch the next tile's halo values when its stage has already
        // landed (never wait for it here); the loads stay in flight while
        // this tile is computed
        pref = false;
        if (tid < a.nring && Tg + G < a.NT) {
            const int sn = (s + 1 == a.nstage) ? 0 : s + 1;
            const uint32_t pn = (sn == 0) ? parity ^ 1u : parity;
            if (mbar_test(&bars[sn], pn)) {
                const TileRef tn_ref = resolve<MULTI>(a, in, out, Tg + G);
                const int32_t *nrow_n = reinterpret_cast<const int32_t *>(smem + sn * a.stage_bytes);
#pragma unroll
                for (int k = 0; k < kRingRegs; ++k) {
                    const int e = tid + k * nth;
                    if (e < a.nring) {
                        const uint32_t w0 = __ldg(a.ring + 2 * e);
                        const int32_t tn = nrow_n[w0 >> 24];
                        rv[k] = (tn >= 0) ? tn_ref.in[(int64_t)tn * a.KL + __ldg(a.ring + 2 * e + 1)] : 0u;
                    }
                }
                pref = true;
            }
        }
        if (!DirectStore<Pol>::value && tid == 0) bulk_wait_read_all();   // previous tile's bulk store has read ostage
        __syncthreads();
        // stage s is consumed (policies that compute from the stage itself
        // refill it after the compute): refill it with the tile nstage
        // iterations ahead
        if (!Pol::kRingInTile && tid == 0) {
            const int64_t Tn = Tg + a.nstage * G;
            fence_proxy_async_smem();
            if (Tn < a.NT) issue_tile(a, resolve<MULTI>(a, in, out, Tn), stage, &bars[s]);
        }
        Pol::compute(a, io, box, tab, R);
        __syncthreads();
        if (Pol::kRingInTile && tid == 0) {
            const int64_t Tn = Tg + a.nstage * G;
            fence_proxy_async_smem();
            if (Tn < a.NT) issue_tile(a, resolve<MULTI>(a, in, out, Tn), stage, &bars[s]);
        }
        if constexpr (DirectStore<Pol>::value) continue;   // the compute wrote the results
        uint8_t *tout = ostage + io.a_out;
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

template <int DIM, int MODE, bool MULTI>
__global__ void __launch_bounds__(256, MODE == kModeTap || MODE == kModeRows0 || MODE == kModeRows1 || MODE == kModeLid1 || MODE == kModeBox3 ? 3 : 4)
step_tma_kernel(FracDev F, StepArgs a, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    using Pol = typename PolicyOf<DIM, MODE>::type;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + a.off_bar);
    uint8_t *box = smem + a.off_box;
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + a.off_tab);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t G = gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
        fence_proxy_async_smem();
    }
    if constexpr (Pol::kRingInTile) {
        if constexpr (Pol::kPadded) {
            // the all-zero unit of every stage (no copy ever writes it)
            for (int s = 0; s < a.nstage; ++s)
                for (int j = tid; j < Pol::NB; j += nth)
                    smem[s * a.stage_bytes + 4 * a.nbrw + kStagePad + a.zoff + j] = 0;
        }
        if (Pol::kPadded) __syncthreads();   // every warp issues: the barriers must be initialised
        if (Pol::kPadded || tid < 32) {
            __syncwarp();
            for (int s = 0; s < a.nstage; ++s) {
                const int64_t Tg = blockIdx.x + s * G;
                if (Tg < a.NT) issue_stage<MULTI, Pol>(a, resolve<MULTI>(a, in, out, Tg), smem + s * a.stage_bytes, &bars[s]);
            }
        }
    } else if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) {
            const int64_t Tg = blockIdx.x + s * G;
            if (Tg < a.NT) issue_tile(a, resolve<MULTI>(a, in, out, Tg), smem + s * a.stage_bytes, &bars[s]);
        }
    }
    for (int i = tid; i < a.box_bytes / 16; i += nth)
        reinterpret_cast<uint4 *>(box)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < a.ntab; i += nth) tab[i] = a.tab[i];
    __syncthreads();

    typename Pol::Regs R;
    Pol::init(a, R);
    if constexpr (Pol::kRingInTile)
        one_barrier_loop<MULTI, Pol>(a, in, out, smem, bars, tab, R);
    else
        staged_loop<MULTI, Pol>(a, in, out, smem, bars, box, tab, R);
}

// Byte tables of the rule for the quad policy (see rule4).
static void rule_tables(uint32_t birth, uint32_t survive, uint32_t lut[4])
{
    uint8_t dead[8], live[8];
    for (int j = 0; j < 8; ++j) {
        // dead cell: total = live neighbours (<= 8)
        uint8_t d = (birth >> j) & 1u;
        if (j + 8 <= 8 && ((birth >> (j + 8)) & 1u)) d |= 0x80;
        // live cell: total = live neighbours + 1 (1..9)
        uint8_t l = (j >= 1) ? ((survive >> (j - 1)) & 1u) : 0u;
        if (j + 8 <= 9 && ((survive >> (j + 7)) & 1u)) l |= 0x80;
        dead[j] = d;
        live[j] = l;
    }
    lut[0] = dead[0] | dead[1] << 8 | dead[2] << 16 | (uint32_t)dead[3] << 24;
    lut[1] = dead[4] | dead[5] << 8 | dead[6] << 16 | (uint32_t)dead[7] << 24;
    lut[2] = live[0] | live[1] << 8 | live[2] << 16 | (uint32_t)live[3] << 24;
    lut[3] = live[4] | live[5] << 8 | live[6] << 16 | (uint32_t)live[7] << 24;
}

void make_rule(uint32_t birth, uint32_t survive, Rule *r)
{
    r->birth = birth;
    r->survive = survive;
    rule_tables(birth, survive, r->lut);
    // byte j: bit 0 = a dead cell with j live neighbours is born, bit 7 = a
    // live cell with total j (j - 1 live neighbours) survives
    uint8_t sp[8];
    for (int j = 0; j < 8; ++j)
        sp[j] = (uint8_t)(((birth >> j) & 1u) | (j >= 1 ? ((survive >> (j - 1)) & 1u) << 7 : 0u));
    r->lut_sparse[0] = sp[0] | sp[1] << 8 | sp[2] << 16 | (uint32_t)sp[3] << 24;
    r->lut_sparse[1] = sp[4] | sp[5] << 8 | sp[6] << 16 | (uint32_t)sp[7] << 24;
}

static void fill_args(const fractal *f, StepArgs &a)
{
    const StepPlan &p = f->plan;
    a.KL = p.KL;
    a.NT = p.NT;
    a.tile0 = 0;
    a.cells = f->cells;
    a.Px = p.Px;
    a.Py = p.Py;
    a.nring = p.nring;
    a.nhalo = p.nhalo;
    a.hbytes = p.hbytes;
    a.zoff = p.zoff;
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
    a.tapz = p.tapz;
    a.nq = p.nq;
    a.wait_limit = kWaitLimit;
    a.extra_tx = 0;
    a.tab = p.pos;
    a.ring = p.ring;
    a.nbr = p.nbr;
    a.status = f->status;
    a.tile_inst = nullptr;
    a.insts = nullptr;
    a.gen = 0;
    for (int q = 0; q < kMaxGroup; ++q) {
        a.lid_of_q[q] = p.lid_of_q[q];
        a.rel_of_lid[q] = p.rel_of_lid[q];
    }
    for (int q = 0; q < 8; ++q) a.row_sel[q] = p.row_sel[q];
    for (int q = 0; q < 9; ++q) a.pack_sel[q] = p.pack_sel[q];
    a.b3 = p.b3;
}

template <bool MULTI>
static int dispatch(const fractal *f, const StepArgs &a, int grid, const uint8_t *in, uint8_t *out,
                    cudaStream_t st)
{
    const StepPlan &p = f->plan;
    if (p.mode == kModeBit3) {
        // a warp per tile; the B5/S45 rule with constants where the launch has one rule
        // and the Menger sponge's five words per block with constants
        grid = (int)std::min<int64_t>(grid, (a.NT + kB3Warps - 1) / kB3Warps);
        const bool b5s45 = !MULTI && a.rule.birth == (1u << 5) && a.rule.survive == ((1u << 4) | (1u << 5));
        if (p.b3.k != 20 && b5s45)
            step_bit3_kernel<MULTI, !MULTI, 0, false, false><<<grid, p.block, p.smem, st>>>(a, in, out);
        else if (p.b3.k != 20)
            step_bit3_kernel<MULTI, false, 0, false, false><<<grid, p.block, p.smem, st>>>(a, in, out);
        else if (b5s45)
            step_bit3_kernel<MULTI, !MULTI, 5, false, false><<<grid, p.block, p.smem, st>>>(a, in, out);
        else
            step_bit3_kernel<MULTI, false, 5, false, false><<<grid, p.block, p.smem, st>>>(a, in, out);
        FR_CUDA(cudaGetLastError());
        return FR_OK;
    }
    if (f->dim == 3 && p.mode == kModeBox3)
        step_tma_kernel<3, kModeBox3, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (f->dim == 3)
        step_tma_kernel<3, kModeCell, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeQuad)
        step_tma_kernel<2, kModeQuad, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeTap)
        step_tma_kernel<2, kModeTap, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeRows0)
        step_tma_kernel<2, kModeRows0, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeRows1)
        step_tma_kernel<2, kModeRows1, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeLid1)
        step_tma_kernel<2, kModeLid1, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeGroup4)
        step_tma_kernel<2, kModeGroup4, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else if (p.mode == kModeGroup3)
        step_tma_kernel<2, kModeGroup3, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    else
        step_tma_kernel<2, kModeCell, MULTI><<<grid, p.block, p.smem, st>>>(f->dev, a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

int launch_step_once(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth,
                     uint32_t survive, cudaStream_t st)
{
    StepArgs a;
    fill_args(f, a);
    make_rule(birth, survive, &a.rule);
    if (f->test_extra_tx) {
        // armed by fractal_test_arm_timeout: this launch only
        a.extra_tx = f->test_extra_tx;
        a.wait_limit = f->test_wait_limit;
        f->test_extra_tx = 0;
        f->test_wait_limit = 0;
    }
    return dispatch<false>(f, a, f->plan.grid, in, out, st);
}

int launch_step_range(fractal *f, const uint8_t *in, uint8_t *out, int64_t T0, int64_t T1, uint32_t birth,
                      uint32_t survive, cudaStream_t st)
{
    if (T1 <= T0) return FR_OK;
    StepArgs a;
    fill_args(f, a);
    make_rule(birth, survive, &a.rule);
    a.tile0 = T0;
    a.NT = T1 - T0;
    const int grid = (int)std::min<int64_t>((int64_t)f->plan.per_sm * f->num_sms, a.NT);
    return dispatch<false>(f, a, grid, in, out, st);
}

int launch_step_tiles(fractal *f, const uint8_t *in, uint8_t *out, const int32_t *nbr, int64_t ntiles,
                      int64_t readable_cells, uint32_t birth, uint32_t survive, cudaStream_t st)
{
    if (ntiles <= 0) return FR_OK;
    StepArgs a;
    fill_args(f, a);
    make_rule(birth, survive, &a.rule);
    a.NT = ntiles;
    a.cells = readable_cells;
    a.nbr = nbr;
    const int grid = (int)std::min<int64_t>((int64_t)f->plan.per_sm * f->num_sms, ntiles);
    return dispatch<false>(f, a, grid, in, out, st);
}

bool bit3_plan(const fractal *f) { return f->plan.pos && f->plan.mode == kModeBit3; }

// one generation of a bit3 plan reading / writing bit-packed states
template <bool IB, bool OB>
static int launch_bit3_mode(const fractal *f, const StepArgs &a, const uint8_t *in, uint8_t *out, cudaStream_t st)
{
    const StepPlan &p = f->plan;
    const bool states_only = IB && OB;
    const int grid = (int)std::min<int64_t>(states_only ? p.b3.grid_states : p.grid, (a.NT + kB3Warps - 1) / kB3Warps);
    const int smem = states_only ? bit3_states_smem(p) : p.smem;
    const bool b5s45 = a.rule.birth == (1u << 5) && a.rule.survive == ((1u << 4) | (1u << 5));
    if (p.b3.k != 20 && b5s45)
        step_bit3_kernel<false, true, 0, IB, OB><<<grid, p.block, smem, st>>>(a, in, out);
    else if (p.b3.k != 20)
        step_bit3_kernel<false, false, 0, IB, OB><<<grid, p.block, smem, st>>>(a, in, out);
    else if (b5s45)
        step_bit3_kernel<false, true, 5, IB, OB><<<grid, p.block, smem, st>>>(a, in, out);
    else
        step_bit3_kernel<false, false, 5, IB, OB><<<grid, p.block, smem, st>>>(a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

int launch_bit3_generations(fractal *f, const uint8_t *in, uint8_t *out, int64_t steps, uint32_t birth,
                            uint32_t survive, cudaStream_t st)
{
    if (!bit3_plan(f) || steps < 2) {
        set_error(FR_EINVAL, "fractal_step: bit-packed generations need a bit3 plan and two generations or more");
        return FR_EINVAL;
    }
    const size_t bytes = (size_t)f->plan.NT * kB3StateWords * sizeof(uint32_t);
    for (int i = 0; i < 2; ++i) {
        if (f->b3_state[i]) continue;
        cudaError_t e = cudaMalloc(&f->b3_state[i], bytes);
        if (e != cudaSuccess) {
            f->b3_state[i] = nullptr;
            return cuda_fail(e, "fractal_step: bit-state allocation");
        }
    }
    StepArgs a;
    fill_args(f, a);
    make_rule(birth, survive, &a.rule);
    a.b3.sin = nullptr;
    a.b3.sout = f->b3_state[0];
    int rc = launch_bit3_mode<false, true>(f, a, in, out, st);
    for (int64_t g = 2; g < steps && !rc; ++g) {
        a.b3.sin = f->b3_state[(g - 2) & 1];
        a.b3.sout = f->b3_state[(g - 1) & 1];
        rc = launch_bit3_mode<true, true>(f, a, in, out, st);
    }
    if (!rc) {
        a.b3.sin = f->b3_state[(steps - 2) & 1];
        a.b3.sout = nullptr;
        rc = launch_bit3_mode<true, false>(f, a, in, out, st);
    }
    return rc;
}

int launch_step_multi(const fractal *cls, const InstDesc *descs, const int32_t *tile_inst,
                      int ninst, int64_t total, int gen, cudaStream_t st)
{
    if (ninst <= 0 || total <= 0) return FR_OK;
    StepArgs a;
    fill_args(cls, a);
    make_rule(0, 0, &a.rule);
    a.NT = total;
    a.cells = 0;
    a.nbr = nullptr;
    a.tile_inst = tile_inst;
    a.insts = descs;
    a.gen = gen;
    const int grid = (int)std::min<int64_t>((int64_t)cls->plan.per_sm * cls->num_sms, total);
    return dispatch<true>(cls, a, grid, nullptr, nullptr, st);
}

// ---------------------------------------------------------- temporal blocking

void free_tb_plan(TbPlan &p)
{
    cudaFree(p.upos);
    cudaFree(p.ring);
    cudaFree(p.nbr);
    p = TbPlan();
}

struct TbLayout {
    int W = 0, NWB = 0, RS = 0, nring = 0;
    int off_halo = 0, off_pres = 0, off_box0 = 0, off_box1 = 0, off_mask = 0, total = 0;
};

static TbLayout tb_layout(const fractal *f, int L)
{
    TbLayout y;
    int nus = 1;
    for (int i = 0; i < L - 2; ++i) nus *= 3;
    const int64_t KL = ipow(f->k, L), NB = (int64_t)f->k * f->k;
    y.W = 9 * nus + 18;
    y.NWB = (y.W + 31) / 32;
    y.RS = y.NWB + 2;
    y.nring = 4 * nus + 4;   // at most: the unit ring around the tile's unit grid
    const int64_t boxb = round16(4 * (int64_t)y.W * y.RS);
    int64_t off = round16(KL);
    y.off_halo = (int)off;
    off = round16(off + NB * y.nring + 4);
    y.off_pres = (int)off;
    off = round16(off + y.nring + 4);
    y.off_box0 = (int)off;
    y.off_box1 = (int)(off + boxb);
    y.off_mask = (int)(off + 2 * boxb);
    const int64_t total = off + 3 * boxb;
    y.total = total > (1 << 30) ? (1 << 30) : (int)total;
    return y;
}

int ensure_tb_plan(fractal *f)
{
    const int P = rows_preset_of(f);
    if (P < 0) {
        set_error(FR_EINVAL, "temporal blocking: only the carpet and the Vicsek fractal (preset offsets)");
        return FR_EINVAL;
    }
    int L = f->tb_levels_user;
    if (L < 0) {
        // the deepest tile whose shared memory stays within 100 KB
        L = -1;
        for (int l = 2; l <= std::min(f->r, 6); ++l)
            if (tb_layout(f, l).total <= 100 * 1024 && ipow(f->k, f->r - l) < ((int64_t)1 << 31)) L = l;
    }
    if (L < 2 || L > f->r) {
        set_error(FR_EINVAL, "temporal blocking: needs a tile depth of at least 2 levels");
        return FR_EINVAL;
    }
    if (f->tb.L == L && f->tb.upos) return FR_OK;
    free_tb_plan(f->tb);
    int rc = ensure_status(f);
    if (rc) return rc;
    const TbLayout y = tb_layout(f, L);
    int optin = 0, dev = 0;
    FR_CUDA(cudaGetDevice(&dev));
    FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (y.total > optin) {
        set_error(FR_EINVAL, "temporal blocking: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    TbPlan p;
    p.L = L;
    p.preset = P;
    p.KL = ipow(f->k, L);
    p.NT = ipow(f->k, f->r - L);
    if (p.NT >= ((int64_t)1 << 31)) {
        set_error(FR_EOVERFLOW, "temporal blocking: more than 2^31 tiles at this tile depth");
        return FR_EOVERFLOW;
    }
    int nus = 1, nu = 1;
    for (int i = 0; i < L - 2; ++i) {
        nus *= 3;
        nu *= f->k;
    }
    p.nu = nu;
    // unit grid of a tile (the unit layout of rows_layout.h against the fractal's own lambda)
    std::vector<int> M((size_t)nus * nus, -1);
    std::vector<uint16_t> upos(nu);
    const int NB = f->k * f->k;
    for (int q = 0; q < nu; ++q) {
        int c[3];
        host_lambda(f, q, L - 2, c);
        M[(size_t)c[1] * nus + c[0]] = q;
        upos[q] = (uint16_t)((c[0] + 1) | ((c[1] + 1) << 8));
        for (int u = 0; u < NB; ++u) {
            int d[3];
            host_lambda(f, (int64_t)NB * q + u, L, d);
            const int ex = 9 * c[0] + (P == 0 ? rp_x<0>(u) : rp_x<1>(u));
            const int ey = 9 * c[1] + (P == 0 ? rp_y<0>(u) : rp_y<1>(u));
            if (d[0] != ex || d[1] != ey) {
                set_error(FR_EINVAL, "temporal blocking: unit layout does not match the fractal");
                return FR_EINVAL;
            }
        }
    }
    // the ring of units of the neighbouring tiles around the tile's unit grid
    std::vector<uint32_t> ring;
    for (int by = 0; by < nus + 2; ++by)
        for (int bx = 0; bx < nus + 2; ++bx) {
            if (bx > 0 && bx < nus + 1 && by > 0 && by < nus + 1) continue;
            const int gx = bx - 1, gy = by - 1;
            const int tdx = gx < 0 ? -1 : (gx >= nus ? 1 : 0), tdy = gy < 0 ? -1 : (gy >= nus ? 1 : 0);
            const int lu = M[(size_t)((gy + nus) % nus) * nus + (gx + nus) % nus];
            if (lu < 0) continue;
            const int d9 = (tdx + 1) + 3 * (tdy + 1);
            const int slot = d9 < 4 ? d9 : d9 - 1;
            ring.push_back((uint32_t)lu | ((uint32_t)slot << 24));
            ring.push_back((uint32_t)bx | ((uint32_t)by << 8));
        }
    p.nring = (int)ring.size() / 2;
    if (p.nring > y.nring) {
        set_error(FR_EINVAL, "temporal blocking: halo ring larger than planned");
        return FR_EINVAL;
    }
    p.W = y.W;
    p.RS = y.RS;
    p.NWB = y.NWB;
    p.off_halo = y.off_halo;
    p.off_pres = y.off_pres;
    p.off_box0 = y.off_box0;
    p.off_box1 = y.off_box1;
    p.off_mask = y.off_mask;
    p.smem = y.total;
    p.block = (p.W * p.NWB >= 1024 || nu >= 256) ? 256 : 128;
    FR_CUDA(cudaMalloc(&p.upos, upos.size() * sizeof(uint16_t)));
    FR_CUDA(cudaMemcpy(p.upos, upos.data(), upos.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    FR_CUDA(cudaMalloc(&p.ring, std::max<size_t>(ring.size(), 2) * sizeof(uint32_t)));
    if (!ring.empty())
        FR_CUDA(cudaMemcpy(p.ring, ring.data(), ring.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    cudaError_t e = cudaMalloc(&p.nbr, (size_t)p.NT * 8 * sizeof(int32_t));
    if (e != cudaSuccess) {
        free_tb_plan(p);
        return cuda_fail(e, "temporal blocking: neighbour table allocation");
    }
    {
        const int64_t g = std::min<int64_t>((p.NT + 255) / 256, (int64_t)f->num_sms * 16);
        nbr_table_kernel<<<(int)std::max<int64_t>(g, 1), 256>>>(f->dev, p.NT, f->r - L,
                                                                (int32_t)ipow(f->s, f->r - L), 8, p.nbr);
        FR_CUDA(cudaGetLastError());
        FR_CUDA(cudaDeviceSynchronize());
    }
    auto kfn = P == 0 ? step_tb_kernel<0, false> : step_tb_kernel<1, false>;
    auto kfl = P == 0 ? step_tb_kernel<0, true> : step_tb_kernel<1, true>;
    FR_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FR_CUDA(cudaFuncSetAttribute(kfl, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    int per_sm_life = 0;
    FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p.per_sm, kfn, p.block, p.smem));
    FR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_life, kfl, p.block, p.smem));
    p.per_sm = std::min(p.per_sm, per_sm_life);
    if (p.per_sm < 1) {
        free_tb_plan(p);
        set_error(FR_EINVAL, "temporal blocking: tile does not fit in shared memory");
        return FR_EINVAL;
    }
    p.grid = (int)std::min<int64_t>((int64_t)p.per_sm * f->num_sms, p.NT);
    f->tb = p;
    return FR_OK;
}

int launch_tb_once(fractal *f, const uint8_t *in, uint8_t *out, int gens, uint32_t birth, uint32_t survive,
                   cudaStream_t st)
{
    const TbPlan &p = f->tb;
    TbArgs a;
    a.KL = p.KL;
    a.NT = p.NT;
    a.nu = p.nu;
    a.nring = p.nring;
    a.W = p.W;
    a.RS = p.RS;
    a.NWB = p.NWB;
    a.gens = gens;
    a.birth = birth;
    a.survive = survive;
    a.upos = p.upos;
    a.ring = p.ring;
    a.nbr = p.nbr;
    a.off_halo = p.off_halo;
    a.off_pres = p.off_pres;
    a.off_box0 = p.off_box0;
    a.off_box1 = p.off_box1;
    a.off_mask = p.off_mask;
    a.status = f->status;
    const bool life = birth == 0x8u && survive == 0xCu;   // B3/S23
    if (p.preset == 0 && life)
        step_tb_kernel<0, true><<<p.grid, p.block, p.smem, st>>>(a, in, out);
    else if (p.preset == 0)
        step_tb_kernel<0, false><<<p.grid, p.block, p.smem, st>>>(a, in, out);
    else if (life)
        step_tb_kernel<1, true><<<p.grid, p.block, p.smem, st>>>(a, in, out);
    else
        step_tb_kernel<1, false><<<p.grid, p.block, p.smem, st>>>(a, in, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

// ---------------------------------------------------------------- autotune

static std::mutex g_tune_mu;
static std::map<std::string, std::pair<int, int>> g_tune_cache;  // fractal + device -> (tile levels, stages)

static std::string tune_key(const fractal *f)
{
    cudaDeviceProp prop;
    std::string name = "?";
    if (cudaGetDeviceProperties(&prop, f->device) == cudaSuccess) name = prop.name;
    std::string key = name + "|" + std::to_string(f->k) + "," + std::to_string(f->s) + "," +
                      std::to_string(f->r) + "," + std::to_string(f->dim) + "|";
    for (int32_t v : f->offsets) key += std::to_string(v) + ",";
    if (f->mixed) {
        key += "|levels:";
        for (int32_t v : f->lev_k) key += std::to_string(v) + ",";
    }
    return key;
}

int cached_tile_levels(const fractal *f, int *stages)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(f));
    if (stages) *stages = it == g_tune_cache.end() ? -1 : it->second.second;
    return it == g_tune_cache.end() ? -1 : it->second.first;
}

// Times the candidate plans on the caller's buffers and keeps the fastest:
// the tile depths (the deepest that fit in shared memory and the three
// below), each with 2, 3 and 4 input pipeline stages.
int autotune_step(fractal *f, const uint8_t *in, uint8_t *out, uint32_t birth, uint32_t survive,
                  cudaStream_t st, int *best_out)
{
    int lmax = 0;
    f->stages_user = -1;
    for (int L = 0; L <= f->r; ++L) {
        if (plan_layout(f, L).total > 200 * 1024) break;
        lmax = L;
    }
    int best = -1, best_st = -1;
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    FR_CUDA(cudaEventCreate(&e0));
    FR_CUDA(cudaEventCreate(&e1));
    for (int L = lmax; L >= 0 && L >= lmax - 3; --L) {
        if (cells_above(f, L) >= ((int64_t)1 << 31)) break;
        for (int ns = 2; ns <= 4; ++ns) {
            f->tile_levels_user = L;
            f->stages_user = ns;
            if (plan_layout(f, L).total > 200 * 1024) continue;
            if (ensure_step_plan(f) != FR_OK) continue;
            if (f->plan.mode == kModeBit3 && ns > 2) continue;   // it has no input stages
            int rc = FR_OK;
            for (int w = 0; w < 2 && !rc; ++w) rc = launch_step_once(f, in, out, birth, survive, st);
            if (!rc) rc = (cudaEventRecord(e0, st) == cudaSuccess) ? FR_OK : FR_ECUDA;
            for (int w = 0; w < 3 && !rc; ++w) rc = launch_step_once(f, in, out, birth, survive, st);
            if (!rc) rc = (cudaEventRecord(e1, st) == cudaSuccess) ? FR_OK : FR_ECUDA;
            if (!rc) rc = (cudaEventSynchronize(e1) == cudaSuccess) ? FR_OK : FR_ECUDA;
            float ms = 0.f;
            if (!rc && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best < 0 || ms < best_ms)) {
                best = L;
                best_st = ns;
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        f->tile_levels_user = -1;
        f->stages_user = -1;
        set_error(FR_EINVAL, "fractal_autotune: no tile depth could be planned");
        return FR_EINVAL;
    }
    f->tile_levels_user = best;
    f->stages_user = best_st;
    int rc = ensure_step_plan(f);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(f)] = std::make_pair(best, best_st);
    }
    if (best_out) *best_out = best;
    return take_status(f);
}

}  // namespace fr
