/*
 * oracle.c -- plain, slow CPU oracle for cellular automata on NBB fractals
 * kept in compact storage (Quezada & Navarro, "Accelerating Compact Fractals
 * with Tensor Core GPUs", 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code.  The library's GPU path never
 * calls it, and the two share no source, header, table or helper.
 *
 * Every function is the textbook definition written out, one level, one
 * neighbour and one cell at a time, in 64-bit integers:
 *
 *   - An NBB fractal F_n^{k,s} (Sec. 1) is given by its transition table
 *     off[j][0..dim-1], j = 0..k-1: level m+1 is k translated copies of level
 *     m, copy j placed at off[j] * s^m.  Level 0 is one cell.  The side of
 *     the bounding box is n = s^r and the compact volume is V = k^r (Eq. 1).
 *   - Membership: a box cell p belongs to the fractal iff, at every level mu,
 *     its base-s digit tuple (floor(p_i / s^mu) mod s)_i is one of the
 *     offsets.  This is decided by linear search, with no lambda or nu.
 *   - nu (Sec. 3.1, Eqs. 2-8): embedded coordinate -> compact index.  At each
 *     level the replica ID H is the row j of the table whose offset equals
 *     the digit tuple (the inverse transition table; the paper's procedural
 *     Eq. 2 is this rule for one orientation of the triangle).  The linear
 *     compact index is omega = sum_mu H_mu k^mu ("canonical order", level 0
 *     least significant).  A tuple that matches no offset means "outside".
 *   - nu2d: the paper's two-dimensional compact coordinate (Eqs. 6-8), with
 *     tau_x(k,mu) = k^floor(mu/2) for even mu and tau_y(k,mu) = k^floor(mu/2)
 *     for odd mu; in 3D the axes cycle x,y,z with k^floor(mu/3).
 *   - lambda (Sec. 3): compact index -> embedded coordinate, the inverse of
 *     nu: p = sum_mu s^mu off[d_mu] with d_mu = floor(omega / k^mu) mod k.
 *   - compact step (Sec. 3, the stencil procedure): for every omega, p =
 *     lambda(omega); for each Moore neighbour q of p (8 in 2D, 26 in 3D)
 *     inside the box, omega' = nu(q); neighbours that are outside the box or
 *     off the fractal are dead; count the live ones; apply the life-like rule
 *     (bit c of `birth` / `survive` = outcome for c live neighbours).  The
 *     update is synchronous: `in` is read, `out` is written.
 *   - bounding-box step (Sec. 4, approach "BB"): the same rule applied to the
 *     whole n^dim byte box (x fastest, then y, then z).  Cells off the fractal
 *     count as dead whatever their byte, and are written as 0.
 *   - a fractal with a different transition table at each level (the
 *     paper's conclusions, future work): the same definitions level by
 *     level with level mu's own table, compact indices in mixed radix
 *     (oracle_mix_*).
 *   - Bernoulli initial state: the omega-th output of SplitMix64 (Steele, Lea
 *     & Flood 2014) seeded with `seed`, i.e. mix(seed + (omega+1) * gamma);
 *     alive iff its top 53 bits are below floor(p * 2^53).  Not part of the
 *     paper: it only makes seeded synthetic inputs.
 *
 * Loops over cells carry an OpenMP pragma so that the benchmark can time the
 * oracle on all host cores; the per-cell code is the same either way.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXDIM 3

/* ------------------------------------------------------------------ basics */

int64_t oracle_ipow(int64_t b, int e)
{
    int64_t v = 1;
    for (int i = 0; i < e; ++i) v *= b;
    return v;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Replica ID at one level: the row j of the transition table equal to the
 * digit tuple t, or -1 if no row matches (Sec. 3.1, the helper H). */
static int replica_id(int k, int dim, const int32_t *off, const int64_t *t)
{
    for (int j = 0; j < k; ++j) {
        int same = 1;
        for (int i = 0; i < dim; ++i)
            if ((int64_t)off[j * dim + i] != t[i]) same = 0;
        if (same) return j;
    }
    return -1;
}

static int in_box(int s, int r, int dim, const int64_t *p)
{
    int64_t n = oracle_ipow(s, r);
    for (int i = 0; i < dim; ++i)
        if (p[i] < 0 || p[i] >= n) return 0;
    return 1;
}

/* ----------------------------------------------------- membership (brute) */

int oracle_is_member(int k, int s, int r, int dim, const int32_t *off,
                     const int64_t *p)
{
    if (!in_box(s, r, dim, p)) return 0;
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        if (replica_id(k, dim, off, t) < 0) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------ lambda, nu */

void oracle_lambda(int k, int s, int r, int dim, const int32_t *off,
                   int64_t omega, int64_t *p)
{
    for (int i = 0; i < dim; ++i) p[i] = 0;
    for (int mu = 0; mu < r; ++mu) {
        int64_t d = (omega / oracle_ipow(k, mu)) % k;
        int64_t smu = oracle_ipow(s, mu);
        for (int i = 0; i < dim; ++i) p[i] += smu * off[d * dim + i];
    }
}

int64_t oracle_nu(int k, int s, int r, int dim, const int32_t *off,
                  const int64_t *p)
{
    if (!in_box(s, r, dim, p)) return -1;
    int64_t omega = 0;
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        int h = replica_id(k, dim, off, t);
        if (h < 0) return -1;
        omega += (int64_t)h * oracle_ipow(k, mu);
    }
    return omega;
}

/* Eqs. 6-8: c_axis = sum_mu tau_axis(k,mu) * H(mu), tau nonzero only on the
 * axis mu mod dim, with magnitude k^floor(mu/dim).  Returns 0 on success,
 * -1 if p is outside (then c is left at -1). */
int oracle_nu2d(int k, int s, int r, int dim, const int32_t *off,
                const int64_t *p, int64_t *c)
{
    for (int i = 0; i < dim; ++i) c[i] = 0;
    if (!in_box(s, r, dim, p)) {
        for (int i = 0; i < dim; ++i) c[i] = -1;
        return -1;
    }
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        int h = replica_id(k, dim, off, t);
        if (h < 0) {
            for (int i = 0; i < dim; ++i) c[i] = -1;
            return -1;
        }
        int axis = mu % dim;
        c[axis] += (int64_t)h * oracle_ipow(k, mu / dim);
    }
    return 0;
}

/* ------------------------------------------------------------ batch maps */

void oracle_lambda_batch(int k, int s, int r, int dim, const int32_t *off,
                         const int64_t *omega, int64_t count, int64_t *coords)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        oracle_lambda(k, s, r, dim, off, omega[e], coords + e * dim);
}

void oracle_nu_batch(int k, int s, int r, int dim, const int32_t *off,
                     const int64_t *coords, int64_t count, int64_t *omega)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        omega[e] = oracle_nu(k, s, r, dim, off, coords + e * dim);
}

void oracle_nu2d_batch(int k, int s, int r, int dim, const int32_t *off,
                       const int64_t *coords, int64_t count, int64_t *c)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        oracle_nu2d(k, s, r, dim, off, coords + e * dim, c + e * dim);
}

void oracle_member_batch(int k, int s, int r, int dim, const int32_t *off,
                         const int64_t *coords, int64_t count, uint8_t *m)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        m[e] = (uint8_t)oracle_is_member(k, s, r, dim, off, coords + e * dim);
}

/* --------------------------------------------------------------- the rule */

static uint8_t life_rule(int alive, int count, uint32_t birth, uint32_t survive)
{
    uint32_t mask = alive ? survive : birth;
    return (uint8_t)((mask >> count) & 1u);
}

/* Moore offset number q (0 .. 3^dim - 1) as a vector in {-1,0,1}^dim. */
static void moore_offset(int dim, int q, int64_t *delta)
{
    for (int i = 0; i < dim; ++i) {
        delta[i] = (int64_t)(q % 3) - 1;
        q /= 3;
    }
}

static int is_zero_offset(int dim, const int64_t *delta)
{
    for (int i = 0; i < dim; ++i)
        if (delta[i] != 0) return 0;
    return 1;
}

/* ---------------------------------------------------------- compact step */

/* New state of compact cell omega from the compact state `in` (Sec. 3). */
uint8_t oracle_compact_cell(int k, int s, int r, int dim, const int32_t *off,
                            const uint8_t *in, int64_t omega,
                            uint32_t birth, uint32_t survive)
{
    int64_t p[OR_MAXDIM], q[OR_MAXDIM], delta[OR_MAXDIM];
    oracle_lambda(k, s, r, dim, off, omega, p);
    int nq = 1;
    for (int i = 0; i < dim; ++i) nq *= 3;
    int count = 0;
    for (int e = 0; e < nq; ++e) {
        moore_offset(dim, e, delta);
        if (is_zero_offset(dim, delta)) continue;
        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];
        if (!in_box(s, r, dim, q)) continue;
        int64_t w = oracle_nu(k, s, r, dim, off, q);
        if (w < 0) continue;
        if (in[w] != 0) ++count;
    }
    return life_rule(in[omega] != 0, count, birth, survive);
}

/* out[omega] for omega in [w0, w1). */
void oracle_step_compact_range(int k, int s, int r, int dim, const int32_t *off,
                               const uint8_t *in, uint8_t *out,
                               uint32_t birth, uint32_t survive,
                               int64_t w0, int64_t w1)
{
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t w = w0; w < w1; ++w)
        out[w] = oracle_compact_cell(k, s, r, dim, off, in, w, birth, survive);
}

/* vals[e] = new state of cell omegas[e]. */
void oracle_step_compact_cells(int k, int s, int r, int dim, const int32_t *off,
                               const uint8_t *in, const int64_t *omegas,
                               int64_t count, uint32_t birth, uint32_t survive,
                               uint8_t *vals)
{
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t e = 0; e < count; ++e)
        vals[e] = oracle_compact_cell(k, s, r, dim, off, in, omegas[e],
                                      birth, survive);
}

/* `steps` synchronous generations from `in`, final state in `out`. */
int oracle_run_compact(int k, int s, int r, int dim, const int32_t *off,
                       const uint8_t *in, uint8_t *out, int64_t steps,
                       uint32_t birth, uint32_t survive)
{
    int64_t V = oracle_ipow(k, r);
    uint8_t *a = (uint8_t *)malloc((size_t)V);
    uint8_t *b = (uint8_t *)malloc((size_t)V);
    if (!a || !b) { free(a); free(b); return -1; }
    for (int64_t w = 0; w < V; ++w) a[w] = in[w] != 0;
    for (int64_t t = 0; t < steps; ++t) {
        oracle_step_compact_range(k, s, r, dim, off, a, b, birth, survive, 0, V);
        uint8_t *x = a; a = b; b = x;
    }
    memcpy(out, a, (size_t)V);
    free(a);
    free(b);
    return 0;
}

/* State of cell omega after t generations from `init`, by the recursive
 * definition of a synchronous update (exponential: small t only). */
uint8_t oracle_cell_after(int k, int s, int r, int dim, const int32_t *off,
                          const uint8_t *init, int64_t omega, int t,
                          uint32_t birth, uint32_t survive)
{
    if (t == 0) return init[omega] != 0;
    int64_t p[OR_MAXDIM], q[OR_MAXDIM], delta[OR_MAXDIM];
    oracle_lambda(k, s, r, dim, off, omega, p);
    int nq = 1;
    for (int i = 0; i < dim; ++i) nq *= 3;
    int count = 0;
    for (int e = 0; e < nq; ++e) {
        moore_offset(dim, e, delta);
        if (is_zero_offset(dim, delta)) continue;
        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];
        int64_t w = oracle_nu(k, s, r, dim, off, q);
        if (w < 0) continue;
        count += oracle_cell_after(k, s, r, dim, off, init, w, t - 1,
                                   birth, survive);
    }
    int alive = oracle_cell_after(k, s, r, dim, off, init, omega, t - 1,
                                  birth, survive);
    return life_rule(alive, count, birth, survive);
}

void oracle_cells_after(int k, int s, int r, int dim, const int32_t *off,
                        const uint8_t *init, const int64_t *omegas,
                        int64_t count, int t, uint32_t birth, uint32_t survive,
                        uint8_t *vals)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < count; ++e)
        vals[e] = oracle_cell_after(k, s, r, dim, off, init, omegas[e], t,
                                    birth, survive);
}

/* ------------------------------------------------------ bounding-box step */

static int64_t box_index(int64_t n, int dim, const int64_t *p)
{
    int64_t idx = 0;
    for (int i = dim - 1; i >= 0; --i) idx = idx * n + p[i];
    return idx;
}

static void box_coords(int64_t n, int dim, int64_t idx, int64_t *p)
{
    for (int i = 0; i < dim; ++i) {
        p[i] = idx % n;
        idx /= n;
    }
}

uint8_t oracle_bb_cell(int k, int s, int r, int dim, const int32_t *off,
                       const uint8_t *box, int64_t idx,
                       uint32_t birth, uint32_t survive)
{
    int64_t n = oracle_ipow(s, r);
    int64_t p[OR_MAXDIM], q[OR_MAXDIM], delta[OR_MAXDIM];
    box_coords(n, dim, idx, p);
    if (!oracle_is_member(k, s, r, dim, off, p)) return 0;
    int nq = 1;
    for (int i = 0; i < dim; ++i) nq *= 3;
    int count = 0;
    for (int e = 0; e < nq; ++e) {
        moore_offset(dim, e, delta);
        if (is_zero_offset(dim, delta)) continue;
        for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];
        if (!oracle_is_member(k, s, r, dim, off, q)) continue;
        if (box[box_index(n, dim, q)] != 0) ++count;
    }
    return life_rule(box[idx] != 0, count, birth, survive);
}

void oracle_step_bb(int k, int s, int r, int dim, const int32_t *off,
                    const uint8_t *box_in, uint8_t *box_out,
                    uint32_t birth, uint32_t survive)
{
    int64_t total = oracle_ipow(oracle_ipow(s, r), dim);
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t idx = 0; idx < total; ++idx)
        box_out[idx] = oracle_bb_cell(k, s, r, dim, off, box_in, idx,
                                      birth, survive);
}

void oracle_step_bb_cells(int k, int s, int r, int dim, const int32_t *off,
                          const uint8_t *box_in, const int64_t *idxs,
                          int64_t count, uint32_t birth, uint32_t survive,
                          uint8_t *vals)
{
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t e = 0; e < count; ++e)
        vals[e] = oracle_bb_cell(k, s, r, dim, off, box_in, idxs[e],
                                 birth, survive);
}

int oracle_run_bb(int k, int s, int r, int dim, const int32_t *off,
                  const uint8_t *in, uint8_t *out, int64_t steps,
                  uint32_t birth, uint32_t survive)
{
    int64_t total = oracle_ipow(oracle_ipow(s, r), dim);
    uint8_t *a = (uint8_t *)malloc((size_t)total);
    uint8_t *b = (uint8_t *)malloc((size_t)total);
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, in, (size_t)total);
    if (steps == 0) {
        /* zero generations: the masked box itself */
        #pragma omp parallel for schedule(static)
        for (int64_t idx = 0; idx < total; ++idx) {
            int64_t p[OR_MAXDIM];
            box_coords(oracle_ipow(s, r), dim, idx, p);
            a[idx] = oracle_is_member(k, s, r, dim, off, p) && in[idx] != 0;
        }
    }
    for (int64_t t = 0; t < steps; ++t) {
        oracle_step_bb(k, s, r, dim, off, a, b, birth, survive);
        uint8_t *x = a; a = b; b = x;
    }
    memcpy(out, a, (size_t)total);
    free(a);
    free(b);
    return 0;
}

/* ------------------------------------------------- compact <-> box views */

void oracle_scatter(int k, int s, int r, int dim, const int32_t *off,
                    const uint8_t *compact, uint8_t *box)
{
    int64_t n = oracle_ipow(s, r);
    int64_t total = oracle_ipow(n, dim);
    int64_t V = oracle_ipow(k, r);
    memset(box, 0, (size_t)total);
    #pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < V; ++w) {
        int64_t p[OR_MAXDIM];
        oracle_lambda(k, s, r, dim, off, w, p);
        box[box_index(n, dim, p)] = compact[w] != 0;
    }
}

void oracle_gather(int k, int s, int r, int dim, const int32_t *off,
                   const uint8_t *box, uint8_t *compact)
{
    int64_t n = oracle_ipow(s, r);
    int64_t V = oracle_ipow(k, r);
    #pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < V; ++w) {
        int64_t p[OR_MAXDIM];
        oracle_lambda(k, s, r, dim, off, w, p);
        compact[w] = box[box_index(n, dim, p)] != 0;
    }
}

/* ------------------------------------------------------- seeded init */

/* One SplitMix64 output for the state value z (Steele, Lea & Flood 2014). */
uint64_t oracle_splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* The i-th output (i = 0, 1, ...) of SplitMix64 started from `seed`. */
uint64_t oracle_splitmix64_nth(uint64_t seed, uint64_t i)
{
    return oracle_splitmix64_mix(seed + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

uint64_t oracle_bernoulli_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 53;
    return (uint64_t)(p * 9007199254740992.0); /* floor(p * 2^53) */
}

/* state[w] for w in [w0, w1). */
void oracle_init_bernoulli(uint64_t seed, double p, uint8_t *state,
                           int64_t w0, int64_t w1)
{
    uint64_t thr = oracle_bernoulli_threshold(p);
    #pragma omp parallel for schedule(static)
    for (int64_t w = w0; w < w1; ++w)
        state[w] = (oracle_splitmix64_nth(seed, (uint64_t)w) >> 11) < thr;
}

/* ------------------------------------------- different tables per level */

/* A fractal combined from a different NBB transition table at each scale
 * level (the construction the paper's conclusions propose as future work):
 * level mu (mu = 0 the finest) has ks[mu] replicas whose offsets are the
 * ks[mu] x dim rows starting at offs + dim * (ks[0] + ... + ks[mu-1]); the
 * growth ratio s and the dimension are common to all levels.  The cells
 * number prod_mu ks[mu]; a compact index is the mixed-radix number
 * omega = sum_mu d_mu * (ks[0] * ... * ks[mu-1]), d_mu the replica ID at
 * level mu.  With the same table at every level this is the fractal above. */

static const int32_t *mix_table(int dim, const int32_t *ks, const int32_t *offs, int mu)
{
    int64_t base = 0;
    for (int nu = 0; nu < mu; ++nu) base += ks[nu];
    return offs + dim * base;
}

int64_t oracle_mix_cells(int r, const int32_t *ks)
{
    int64_t v = 1;
    for (int mu = 0; mu < r; ++mu) v *= ks[mu];
    return v;
}

int oracle_mix_is_member(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                         const int64_t *p)
{
    if (!in_box(s, r, dim, p)) return 0;
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        if (replica_id(ks[mu], dim, mix_table(dim, ks, offs, mu), t) < 0) return 0;
    }
    return 1;
}

void oracle_mix_lambda(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                       int64_t omega, int64_t *p)
{
    for (int i = 0; i < dim; ++i) p[i] = 0;
    int64_t weight = 1;   /* ks[0] * ... * ks[mu-1] */
    for (int mu = 0; mu < r; ++mu) {
        int64_t d = (omega / weight) % ks[mu];
        const int32_t *off = mix_table(dim, ks, offs, mu);
        int64_t smu = oracle_ipow(s, mu);
        for (int i = 0; i < dim; ++i) p[i] += smu * off[d * dim + i];
        weight *= ks[mu];
    }
}

int64_t oracle_mix_nu(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                      const int64_t *p)
{
    if (!in_box(s, r, dim, p)) return -1;
    int64_t omega = 0, weight = 1;
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        int h = replica_id(ks[mu], dim, mix_table(dim, ks, offs, mu), t);
        if (h < 0) return -1;
        omega += (int64_t)h * weight;
        weight *= ks[mu];
    }
    return omega;
}

/* The compact coordinate of Eqs. 6-8 for per-level tables: level mu adds
 * H_mu times the product of ks[nu] over the earlier levels nu of the same
 * axis (nu < mu, nu = mu mod dim) to axis mu mod dim. */
int oracle_mix_nu2d(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                    const int64_t *p, int64_t *c)
{
    int64_t weight[OR_MAXDIM];
    for (int i = 0; i < dim; ++i) {
        c[i] = 0;
        weight[i] = 1;
    }
    if (!in_box(s, r, dim, p)) {
        for (int i = 0; i < dim; ++i) c[i] = -1;
        return -1;
    }
    for (int mu = 0; mu < r; ++mu) {
        int64_t smu = oracle_ipow(s, mu);
        int64_t t[OR_MAXDIM];
        for (int i = 0; i < dim; ++i) t[i] = (p[i] / smu) % s;
        int h = replica_id(ks[mu], dim, mix_table(dim, ks, offs, mu), t);
        if (h < 0) {
            for (int i = 0; i < dim; ++i) c[i] = -1;
            return -1;
        }
        int axis = mu % dim;
        c[axis] += (int64_t)h * weight[axis];
        weight[axis] *= ks[mu];
    }
    return 0;
}

void oracle_mix_lambda_batch(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                             const int64_t *omega, int64_t count, int64_t *coords)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        oracle_mix_lambda(s, r, dim, ks, offs, omega[e], coords + e * dim);
}

void oracle_mix_nu_batch(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                         const int64_t *coords, int64_t count, int64_t *omega)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        omega[e] = oracle_mix_nu(s, r, dim, ks, offs, coords + e * dim);
}

void oracle_mix_nu2d_batch(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                           const int64_t *coords, int64_t count, int64_t *c)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        oracle_mix_nu2d(s, r, dim, ks, offs, coords + e * dim, c + e * dim);
}

void oracle_mix_member_batch(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                             const int64_t *coords, int64_t count, uint8_t *m)
{
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e)
        m[e] = (uint8_t)oracle_mix_is_member(s, r, dim, ks, offs, coords + e * dim);
}

/* One synchronous generation of the compact state (Sec. 3 stencil procedure
 * through the per-level lambda and nu). */
void oracle_mix_step(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                     const uint8_t *in, uint8_t *out, uint32_t birth, uint32_t survive)
{
    int64_t V = oracle_mix_cells(r, ks);
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t w = 0; w < V; ++w) {
        int64_t p[OR_MAXDIM], q[OR_MAXDIM], delta[OR_MAXDIM];
        oracle_mix_lambda(s, r, dim, ks, offs, w, p);
        int nq = 1;
        for (int i = 0; i < dim; ++i) nq *= 3;
        int count = 0;
        for (int e = 0; e < nq; ++e) {
            moore_offset(dim, e, delta);
            if (is_zero_offset(dim, delta)) continue;
            for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];
            int64_t n = oracle_mix_nu(s, r, dim, ks, offs, q);
            if (n >= 0 && in[n] != 0) ++count;
        }
        out[w] = life_rule(in[w] != 0, count, birth, survive);
    }
}

/* One generation on the whole box with the per-level membership (cells off
 * the fractal are dead and written 0). */
void oracle_mix_step_bb(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                        const uint8_t *box, uint8_t *out, uint32_t birth, uint32_t survive)
{
    int64_t n = oracle_ipow(s, r), N = oracle_ipow(n, dim);
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t idx = 0; idx < N; ++idx) {
        int64_t p[OR_MAXDIM], q[OR_MAXDIM], delta[OR_MAXDIM];
        box_coords(n, dim, idx, p);
        if (!oracle_mix_is_member(s, r, dim, ks, offs, p)) {
            out[idx] = 0;
            continue;
        }
        int nq = 1;
        for (int i = 0; i < dim; ++i) nq *= 3;
        int count = 0;
        for (int e = 0; e < nq; ++e) {
            moore_offset(dim, e, delta);
            if (is_zero_offset(dim, delta)) continue;
            for (int i = 0; i < dim; ++i) q[i] = p[i] + delta[i];
            if (!oracle_mix_is_member(s, r, dim, ks, offs, q)) continue;
            if (box[box_index(n, dim, q)] != 0) ++count;
        }
        out[idx] = life_rule(box[idx] != 0, count, birth, survive);
    }
}

static int mix_run(int bb, int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                   const uint8_t *in, uint8_t *out, int64_t steps, uint32_t birth, uint32_t survive)
{
    int64_t V = bb ? oracle_ipow(oracle_ipow(s, r), dim) : oracle_mix_cells(r, ks);
    uint8_t *a = (uint8_t *)malloc((size_t)V);
    uint8_t *b = (uint8_t *)malloc((size_t)V);
    if (!a || !b) { free(a); free(b); return -1; }
    for (int64_t w = 0; w < V; ++w) a[w] = in[w] != 0;
    if (bb) {
        /* zero generations still mask the box */
        int64_t n = oracle_ipow(s, r);
        for (int64_t idx = 0; idx < V; ++idx) {
            int64_t p[OR_MAXDIM];
            box_coords(n, dim, idx, p);
            if (!oracle_mix_is_member(s, r, dim, ks, offs, p)) a[idx] = 0;
        }
    }
    for (int64_t t = 0; t < steps; ++t) {
        if (bb) oracle_mix_step_bb(s, r, dim, ks, offs, a, b, birth, survive);
        else oracle_mix_step(s, r, dim, ks, offs, a, b, birth, survive);
        uint8_t *x = a; a = b; b = x;
    }
    memcpy(out, a, (size_t)V);
    free(a);
    free(b);
    return 0;
}

int oracle_mix_run(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                   const uint8_t *in, uint8_t *out, int64_t steps, uint32_t birth, uint32_t survive)
{
    return mix_run(0, s, r, dim, ks, offs, in, out, steps, birth, survive);
}

int oracle_mix_run_bb(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                      const uint8_t *in, uint8_t *out, int64_t steps, uint32_t birth, uint32_t survive)
{
    return mix_run(1, s, r, dim, ks, offs, in, out, steps, birth, survive);
}

/* box[lambda(omega)] = compact[omega] != 0, 0 off the fractal; and back. */
void oracle_mix_scatter(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                        const uint8_t *compact, uint8_t *box)
{
    int64_t n = oracle_ipow(s, r), V = oracle_mix_cells(r, ks);
    memset(box, 0, (size_t)oracle_ipow(n, dim));
    for (int64_t w = 0; w < V; ++w) {
        int64_t p[OR_MAXDIM];
        oracle_mix_lambda(s, r, dim, ks, offs, w, p);
        box[box_index(n, dim, p)] = compact[w] != 0;
    }
}

void oracle_mix_gather(int s, int r, int dim, const int32_t *ks, const int32_t *offs,
                       const uint8_t *box, uint8_t *compact)
{
    int64_t n = oracle_ipow(s, r), V = oracle_mix_cells(r, ks);
    for (int64_t w = 0; w < V; ++w) {
        int64_t p[OR_MAXDIM];
        oracle_mix_lambda(s, r, dim, ks, offs, w, p);
        compact[w] = box[box_index(n, dim, p)] != 0;
    }
}
