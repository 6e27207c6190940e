// maps_tc.cu -- the maps lambda and nu with their level sums on the tensor
// cores (Sec. 3.1, the tensor-core encoding of nu; here exact).
//
// Both maps end in a weighted sum over levels: nu(p) = sum_mu H_mu k^mu and
// the compact coordinate of Eqs. 6-8 = sum_mu H_mu tau(k, mu), lambda(omega)
// = sum_mu s^mu off[d_mu].  Per warp, 32 cells form a 32 x K matrix A of
// small integers (the replica IDs H_mu for nu, the offsets off[d_mu][axis]
// for lambda: one column per level and axis), and the weights form a K x N
// matrix B.  The product is one mma.sync.m16n8k16 (fp16 operands, fp32
// accumulators) per 16 x 8 x 16 block.  To stay exact, every weight is split
// into 11-bit limbs (one column of B per limb: fp16 holds the integers up to
// 2048 exactly) and A's entries are < 256; one fp32 accumulator sums at most
// 32 products (two k-steps), each below 255 * 2047, so it stays below 2^24,
// where fp32 is exact.  Accumulators of further k-steps and the limbs are
// combined as integers.  The per-cell digit decode stays on the CUDA cores.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>

#include "handle.h"

namespace fr {

constexpr int kTcMaxK = 64;     // K (levels x axes), padded to 16
constexpr int kTcCols = 16;     // two n-tiles of 8 columns
constexpr int kTcPitch = 68;    // bytes per row of a warp's A matrix
constexpr int kTcWarps = 4;

struct TcPlan {
    int nk;                        // k-steps of 16
    int ntile;                     // n-tiles of 8 (1 or 2)
    int nout;                      // outputs per cell (lambda: dim; nu: 1 + dim)
    int8_t out_of[kTcCols];        // column -> output, -1 = unused
    int8_t shift_of[kTcCols];      // column -> 11 * limb
    uint16_t w[kTcCols][kTcMaxK];  // limb of each column's weight at each K index
};

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// two bytes b0, b1 (< 1024) as the half2 (b0, b1): the halves 0x6400 | b
// are 1024 + b exactly; 1024 is then subtracted exactly
__device__ __forceinline__ uint32_t bytes_to_half2(uint32_t u16)
{
    uint32_t h;
    asm("prmt.b32 %0, %1, %2, 0x4140;" : "=r"(h) : "r"(u16), "r"(0x64u));
    __half2 v = *reinterpret_cast<__half2 *>(&h);
    v = __hsub2(v, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_half2(uint16_t lo, uint16_t hi)
{
    __half2 v = __halves2half2(__ushort2half_rn(lo), __ushort2half_rn(hi));
    return *reinterpret_cast<uint32_t *>(&v);
}

// B fragments of this lane (column g of each n-tile; K rows 2t, 2t+1, 2t+8,
// 2t+9 of each k-step)
__device__ __forceinline__ void tc_b_frags(const TcPlan &P, uint32_t b[2][4][2])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c = 8 * nt + g, k0 = 16 * kk + 2 * t;
            b[nt][kk][0] = pack_half2(P.w[c][k0], P.w[c][k0 + 1]);
            b[nt][kk][1] = pack_half2(P.w[c][k0 + 8], P.w[c][k0 + 9]);
        }
}

// The 32 x K byte matrix of a warp (rows = its 32 cells) times B; writes
// each cell's outputs (outside cells: -1) through `emit(row, output, value)`
// called by lane 4 g + o for output o of rows g, g + 8, g + 16, g + 24.
template <class Emit>
__device__ __forceinline__ void tc_product(const TcPlan &P, const uint8_t *A, const uint32_t b[2][4][2],
                                           bool outside_mine, Emit emit)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    int64_t acc[4][4];   // [row 16 mt + 8 h + g][output]
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[i][o] = 0;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            if (nt >= P.ntile) continue;
            // accumulate at most two k-steps (32 levels) in fp32, then as integers
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                bool any = false;
#pragma unroll
                for (int kq = 0; kq < 2; ++kq) {
                    const int kk = 2 * kh + kq;
                    if (kk >= P.nk) continue;
                    any = true;
                    const uint8_t *r0 = A + (16 * mt + g) * kTcPitch + 16 * kk + 2 * t;
                    const uint8_t *r1 = r0 + 8 * kTcPitch;
                    uint32_t a[4];
                    a[0] = bytes_to_half2(*reinterpret_cast<const uint16_t *>(r0));
                    a[1] = bytes_to_half2(*reinterpret_cast<const uint16_t *>(r1));
                    a[2] = bytes_to_half2(*reinterpret_cast<const uint16_t *>(r0 + 8));
                    a[3] = bytes_to_half2(*reinterpret_cast<const uint16_t *>(r1 + 8));
                    mma16816(d, a, b[nt][kk]);
                }
                if (!any) continue;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int c = 8 * nt + 2 * t + j;
                    const int o = P.out_of[c];
                    if (o < 0) continue;
                    const int sh = P.shift_of[c];
                    const int64_t v0 = (int64_t)__float2ll_rn(d[j]) << sh;
                    const int64_t v1 = (int64_t)__float2ll_rn(d[2 + j]) << sh;
#pragma unroll
                    for (int oo = 0; oo < 4; ++oo)   // registers, not a runtime-indexed array
                        if (o == oo) {
                            acc[2 * mt][oo] += v0;
                            acc[2 * mt + 1][oo] += v1;
                        }
                }
            }
        }
    // sum each row's outputs over the four lanes of its group
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            if (o >= P.nout) continue;
            acc[i][o] += __shfl_xor_sync(0xffffffffu, acc[i][o], 1);
            acc[i][o] += __shfl_xor_sync(0xffffffffu, acc[i][o], 2);
        }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = 16 * (i >> 1) + 8 * (i & 1) + g;
        const bool out_row = __shfl_sync(0xffffffffu, outside_mine, row);
        int64_t v = acc[i][0];
#pragma unroll
        for (int o = 1; o < 4; ++o)
            if (t == o) v = acc[i][o];
        if (t < P.nout) emit(row, t, out_row ? (int64_t)-1 : v);
    }
}

__global__ void __launch_bounds__(32 * kTcWarps) nu_tc_kernel(FracDev F, TcPlan P, int32_t side,
                                                              const int32_t *__restrict__ coords, int64_t count,
                                                              int64_t *__restrict__ omega,
                                                              int64_t *__restrict__ c2d)
{
    __shared__ __align__(16) uint8_t As[kTcWarps][32 * kTcPitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *A = As[warp];
    for (int i = lane; i < 32 * kTcPitch; i += 32) A[i] = 0;
    uint32_t b[2][4][2];
    tc_b_frags(P, b);
    __syncwarp();
    for (int64_t base = ((int64_t)blockIdx.x * kTcWarps + warp) * 32; base < count;
         base += (int64_t)gridDim.x * kTcWarps * 32) {
        const int64_t e = base + lane;
        bool outside = e >= count;
        uint32_t c[3] = {0, 0, 0};
        if (!outside)
            for (int i = 0; i < F.dim; ++i) {
                const int32_t v = coords[e * F.dim + i];
                if (v < 0 || v >= side) outside = true;
                c[i] = (uint32_t)v;
            }
        // replica ID of every level (Sec. 3.1, H as the inverse table)
        uint8_t *row = A + lane * kTcPitch;
        for (int mu = 0; mu < F.r; ++mu) {
            const uint32_t qx = divu(F.sdiv, c[0]), qy = divu(F.sdiv, c[1]);
            uint32_t t = (c[0] - qx * F.s) + (uint32_t)F.s * (c[1] - qy * F.s);
            c[0] = qx;
            c[1] = qy;
            if (F.dim == 3) {
                const uint32_t qz = divu(F.sdiv, c[2]);
                t += (uint32_t)(F.s * F.s) * (c[2] - qz * F.s);
                c[2] = qz;
            }
            const int h = outside ? 0 : F.hinv[t];
            if (h < 0) outside = true;
            row[mu] = (uint8_t)(h < 0 ? 0 : h);
        }
        __syncwarp();
        tc_product(P, A, b, outside, [&](int r, int o, int64_t v) {
            const int64_t ee = base + r;
            if (ee >= count) return;
            if (o == 0) omega[ee] = v;
            else if (c2d) c2d[ee * F.dim + (o - 1)] = v;
        });
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * kTcWarps) lambda_tc_kernel(FracDev F, TcPlan P,
                                                                  const int64_t *__restrict__ omega,
                                                                  int64_t count, int64_t cells,
                                                                  int32_t *__restrict__ coords)
{
    __shared__ __align__(16) uint8_t As[kTcWarps][32 * kTcPitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *A = As[warp];
    for (int i = lane; i < 32 * kTcPitch; i += 32) A[i] = 0;
    uint32_t b[2][4][2];
    tc_b_frags(P, b);
    __syncwarp();
    for (int64_t base = ((int64_t)blockIdx.x * kTcWarps + warp) * 32; base < count;
         base += (int64_t)gridDim.x * kTcWarps * 32) {
        const int64_t e = base + lane;
        int64_t w = e < count ? omega[e] : -1;
        const bool outside = w < 0 || w >= cells;
        if (outside) w = 0;
        // digits of omega, level mu at columns dim mu .. dim mu + dim - 1
        uint8_t *row = A + lane * kTcPitch;
        uint64_t x = (uint64_t)w;
        for (int mu = 0; mu < F.r; ++mu) {
            uint32_t d;
            if (x < (1ull << 31)) {
                const uint32_t q = (F.k > 1) ? divu(F.kdiv, (uint32_t)x) : (uint32_t)x;
                d = (uint32_t)x - q * (uint32_t)F.k;
                x = q;
            } else {
                const uint64_t q = x / (uint64_t)F.k;
                d = (uint32_t)(x - q * (uint64_t)F.k);
                x = q;
            }
            for (int i = 0; i < F.dim; ++i) row[F.dim * mu + i] = (uint8_t)F.off[d][i];
        }
        __syncwarp();
        tc_product(P, A, b, outside, [&](int r, int o, int64_t v) {
            const int64_t ee = base + r;
            if (ee < count) coords[ee * F.dim + o] = (int32_t)v;
        });
        __syncwarp();
    }
}

static int limbs_for(uint64_t maxval)
{
    int n = 1;
    while (n < 6 && (maxval >> (11 * n)) != 0) ++n;
    return n;
}

static void put_weight(TcPlan &P, int col, int kidx, uint64_t weight, int limb)
{
    P.w[col][kidx] = (uint16_t)((weight >> (11 * limb)) & 2047u);
}

static int tc_fail(const std::string &msg)
{
    set_error(FR_EINVAL, msg);
    return FR_EINVAL;
}

// nu (column block: limbs of k^mu) and the compact coordinate of Eqs. 6-8
// (per axis: limbs of k^floor(mu/dim) on the levels mu = axis mod dim)
static int nu_plan(const fractal *f, TcPlan &P)
{
    if (f->mixed) return tc_fail("fractal_nu_tc: one transition table for every level only");
    memset(&P, 0, sizeof(P));
    for (int c = 0; c < kTcCols; ++c) P.out_of[c] = -1;
    if (f->r > 32) return tc_fail("fractal_nu_tc: more than 32 levels");
    if (f->k > 255) return tc_fail("fractal_nu_tc: k > 255");
    P.nk = (f->r + 15) / 16;
    if (P.nk == 0) P.nk = 1;
    P.nout = 1 + f->dim;
    const int ln = limbs_for((uint64_t)f->cells - 1 > 0 ? (uint64_t)f->cells - 1 : 1);
    int64_t side2 = 1;   // largest compact-coordinate extent: k^ceil(r/dim)
    for (int i = 0; i < (f->r + f->dim - 1) / f->dim; ++i) side2 *= f->k;
    const int l2 = limbs_for((uint64_t)(side2 - 1 > 0 ? side2 - 1 : 1));
    if (ln > 8 || f->dim * l2 > 8) return tc_fail("fractal_nu_tc: level weights too wide");
    P.ntile = 2;
    int64_t km = 1;
    for (int mu = 0; mu < f->r; ++mu) {
        for (int l = 0; l < ln; ++l) put_weight(P, l, mu, (uint64_t)km, l);
        int64_t kd = 1;
        for (int i = 0; i < mu / f->dim; ++i) kd *= f->k;
        const int axis = mu % f->dim;
        for (int l = 0; l < l2; ++l) put_weight(P, 8 + axis * l2 + l, mu, (uint64_t)kd, l);
        km *= f->k;
    }
    for (int l = 0; l < ln; ++l) {
        P.out_of[l] = 0;
        P.shift_of[l] = (int8_t)(11 * l);
    }
    for (int a = 0; a < f->dim; ++a)
        for (int l = 0; l < l2; ++l) {
            P.out_of[8 + a * l2 + l] = (int8_t)(1 + a);
            P.shift_of[8 + a * l2 + l] = (int8_t)(11 * l);
        }
    return FR_OK;
}

// lambda: per axis, limbs of s^mu on the columns of that axis
static int lambda_plan(const fractal *f, TcPlan &P)
{
    if (f->mixed) return tc_fail("fractal_lambda_tc: one transition table for every level only");
    memset(&P, 0, sizeof(P));
    for (int c = 0; c < kTcCols; ++c) P.out_of[c] = -1;
    if (f->dim * f->r > kTcMaxK) return tc_fail("fractal_lambda_tc: dim * r > 64");
    P.nk = (f->dim * f->r + 15) / 16;
    if (P.nk == 0) P.nk = 1;
    P.nout = f->dim;
    const int ls = limbs_for((uint64_t)(f->side - 1 > 0 ? f->side - 1 : 1));
    if (f->dim * ls > 16) return tc_fail("fractal_lambda_tc: coordinates too wide");
    P.ntile = f->dim * ls > 8 ? 2 : 1;
    int64_t sm = 1;
    for (int mu = 0; mu < f->r; ++mu) {
        for (int a = 0; a < f->dim; ++a)
            for (int l = 0; l < ls; ++l) put_weight(P, a * ls + l, f->dim * mu + a, (uint64_t)sm, l);
        sm *= f->s;
    }
    for (int a = 0; a < f->dim; ++a)
        for (int l = 0; l < ls; ++l) {
            P.out_of[a * ls + l] = (int8_t)a;
            P.shift_of[a * ls + l] = (int8_t)(11 * l);
        }
    return FR_OK;
}

static int tc_grid(int64_t count, int num_sms)
{
    int64_t g = (count + 32 * kTcWarps - 1) / (32 * kTcWarps);
    const int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace fr

using namespace fr;

extern "C" int fractal_nu_tc(const fractal_t *f, const int32_t *coords, int64_t count, int64_t *omega,
                             int64_t *compact, void *stream)
{
    clear_error();
    if (!f || (count > 0 && (!coords || !omega))) return tc_fail("fractal_nu_tc: NULL argument");
    if (count < 0) return tc_fail("fractal_nu_tc: count < 0");
    if (count == 0) return FR_OK;
    TcPlan P;
    int rc = nu_plan(f, P);
    if (rc) return rc;
    nu_tc_kernel<<<tc_grid(count, f->num_sms), 32 * kTcWarps, 0, (cudaStream_t)stream>>>(
        f->dev, P, (int32_t)f->side, coords, count, omega, compact);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

extern "C" int fractal_lambda_tc(const fractal_t *f, const int64_t *omega, int64_t count, int32_t *coords,
                                 void *stream)
{
    clear_error();
    if (!f || (count > 0 && (!omega || !coords))) return tc_fail("fractal_lambda_tc: NULL argument");
    if (count < 0) return tc_fail("fractal_lambda_tc: count < 0");
    if (count == 0) return FR_OK;
    TcPlan P;
    int rc = lambda_plan(f, P);
    if (rc) return rc;
    lambda_tc_kernel<<<tc_grid(count, f->num_sms), 32 * kTcWarps, 0, (cudaStream_t)stream>>>(
        f->dev, P, omega, count, f->cells, coords);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}
