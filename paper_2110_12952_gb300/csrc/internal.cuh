// internal.cuh -- shared definitions of the GPU library (not part of the ABI).
//
// The fractal F_n^{k,s} (Sec. 1) is described on the device by FracDev: the
// transition table off[j] and its inverse hinv[digit tuple] (the replica-ID
// helper H of Sec. 3.1, as a look-up table of s^dim entries), plus
// division-by-constant multipliers so that base-s and base-k digit
// extraction costs a multiply-high and a shift instead of a division.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fractal.h"

namespace fr {

constexpr int kMaxSD = 256;     // max s^dim (digit tuples per level)
constexpr int kMaxR = 62;       // max levels stored in tables
constexpr int kMaxDirs = 27;    // 3^dim Moore offsets incl. the centre
constexpr int kTbMaxGenerations = 9;   // temporal blocking: generations per pass (a 9-cell halo)

// Unsigned division of x < 2^31 by a constant d >= 2 (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Thm 4.2
// with N = 31): q = floor(x * m / 2^(31+l)), m = ceil(2^(31+l) / d),
// l = ceil(log2 d).  m fits in 32 bits because d > 2^(l-1).
struct DivU32 {
    uint32_t d, m, sh;  // sh = l - 1 applied after the high 32-bit product
};

inline DivU32 make_div(uint32_t d)
{
    DivU32 r;
    r.d = d;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    if (l == 0) l = 1;  // d == 1 is never used for digits; keep it defined
    unsigned __int128 num = (unsigned __int128)1 << (31 + l);
    uint64_t m = (uint64_t)((num + d - 1) / d);
    r.m = (uint32_t)m;
    r.sh = l - 1;
    return r;
}

__device__ __forceinline__ uint32_t divu(const DivU32 &D, uint32_t x)
{
    return __umulhi(x, D.m) >> D.sh;
}

// One level of a fractal with a different transition table per level
// (fractal_create_mixed): its replica count, division by it, and its table.
struct MixLevel {
    int32_t k;
    DivU32 kdiv;
    int16_t hinv[kMaxSD];
    int8_t off[kMaxSD][3];
};

struct FracDev {
    int32_t k, s, r, dim;
    int32_t sd;          // s^dim
    DivU32 sdiv;         // division by s
    DivU32 kdiv;         // division by k (k >= 2; unused when k == 1)
    int16_t hinv[kMaxSD];  // tuple index t0 + s*t1 + s*s*t2 -> replica id, -1 = none
    int8_t off[kMaxSD][3]; // replica id -> digit tuple
    const MixLevel *mix;   // per-level tables in device memory (r entries), or null: every level as above
};

// digit of omega at a level with k replicas, and omega / k
__device__ __forceinline__ uint32_t mix_digit(const MixLevel &M, uint64_t &omega)
{
    if (omega < (1ull << 31)) {
        const uint32_t q = M.k > 1 ? divu(M.kdiv, (uint32_t)omega) : (uint32_t)omega;
        const uint32_t d = (uint32_t)omega - q * (uint32_t)M.k;
        omega = q;
        return d;
    }
    const uint64_t q = omega / (uint64_t)M.k;
    const uint32_t d = (uint32_t)(omega - q * (uint64_t)M.k);
    omega = q;
    return d;
}

// lambda over levels base .. base + levels - 1 of a fractal with per-level
// tables (coordinates in units of s^base)
__device__ __forceinline__ void lambda_mix(const FracDev &F, uint64_t omega, int levels, int base, int32_t p[3])
{
    int32_t px = 0, py = 0, pz = 0, sm = 1;
    for (int mu = 0; mu < levels; ++mu) {
        const MixLevel &M = F.mix[base + mu];
        const uint32_t d = mix_digit(M, omega);
        px += sm * M.off[d][0];
        py += sm * M.off[d][1];
        pz += sm * M.off[d][2];
        sm *= F.s;
    }
    p[0] = px; p[1] = py; p[2] = pz;
}

// ------------------------------------------------------------ device maps

// lambda over the lowest `levels` levels of `omega` (Sec. 3): coordinates
// p_i = sum_mu s^mu off[d_mu][i].  Requires omega < 2^31 (fast path).
__device__ __forceinline__ void lambda32(const FracDev &F, uint32_t omega, int levels,
                                         int32_t p[3], int base = 0)
{
    if (F.mix) return lambda_mix(F, omega, levels, base, p);
    int32_t px = 0, py = 0, pz = 0, sm = 1;
    for (int mu = 0; mu < levels; ++mu) {
        uint32_t q = (F.k > 1) ? divu(F.kdiv, omega) : omega;
        uint32_t d = omega - q * (uint32_t)F.k;
        omega = q;
        px += sm * F.off[d][0];
        py += sm * F.off[d][1];
        pz += sm * F.off[d][2];
        sm *= F.s;
    }
    p[0] = px; p[1] = py; p[2] = pz;
}

// General lambda for 64-bit omega (levels base .. base + levels - 1; the
// base matters only for per-level tables).
__device__ __forceinline__ void lambda64(const FracDev &F, uint64_t omega, int levels,
                                         int32_t p[3], int base = 0)
{
    if (F.mix) return lambda_mix(F, omega, levels, base, p);
    int32_t px = 0, py = 0, pz = 0, sm = 1;
    int mu = 0;
    for (; mu < levels && omega >= (1ull << 31); ++mu) {
        uint64_t q = omega / (uint64_t)F.k;
        uint32_t d = (uint32_t)(omega - q * (uint64_t)F.k);
        omega = q;
        px += sm * F.off[d][0];
        py += sm * F.off[d][1];
        pz += sm * F.off[d][2];
        sm *= F.s;
    }
    int32_t rest[3];
    lambda32(F, (uint32_t)omega, levels - mu, rest);
    p[0] = px + sm * rest[0];
    p[1] = py + sm * rest[1];
    p[2] = pz + sm * rest[2];
}

// nu over `levels` levels (Sec. 3.1): compact index of the cell at p (all
// coordinates already known to lie in [0, s^levels)), or -1 if some level's
// digit tuple is not a replica.
__device__ __forceinline__ int64_t nu_levels(const FracDev &F, uint32_t x, uint32_t y,
                                             uint32_t z, int levels, int base = 0)
{
    int64_t omega = 0, km = 1;
    if (F.mix) {
        // per-level tables: level base + mu's inverse table and replica count
        for (int mu = 0; mu < levels; ++mu) {
            const MixLevel &M = F.mix[base + mu];
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
            if (h < 0) return -1;
            omega += (int64_t)h * km;
            km *= M.k;
        }
        return omega;
    }
    for (int mu = 0; mu < levels; ++mu) {
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
        if (h < 0) return -1;
        omega += (int64_t)h * km;
        km *= F.k;
    }
    return omega;
}

// ------------------------------------------------------------ host side

void set_error(int code, const std::string &msg);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);

}  // namespace fr

#define FR_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return fr::cuda_fail(_e, #call);         \
    } while (0)
