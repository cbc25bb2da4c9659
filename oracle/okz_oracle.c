/*
 * okz_oracle.c -- plain CPU oracle for the octahedron-model KPZ lattice gas of
 * J. Kelling and G. Odor, "Extremely large scale simulation of a
 * Kardar-Parisi-Zhang model using graphics cards" (arXiv:1110.6745).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the
 * benchmark's CPU legs (its CPU baseline and its reference arm) are the only
 * code allowed to load this library.
 * The CUDA library shares no code with it: no headers, no helpers, no tables.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: one byte per bond, one site at a time, exact integer sums.
 *
 * Representation (Sec. I: "The up edges in the x or y directions are
 * represented by sigma = +1, the down ones by sigma = -1"):
 *   X[y*L + x] = 1  iff  sigma_x(x,y) = h(x+1,y) - h(x,y) = +1, else 0
 *   Y[y*L + x] = 1  iff  sigma_y(x,y) = h(x,y+1) - h(x,y) = +1, else 0
 * Periodic boundaries, L even. H0 = h(0,0) anchors the heights.
 *
 * Readings of the paper taken here (each listed in the design notes):
 *  - Eq. (2) (the generalized Kawasaki rule): the rows of the 2x2 matrices are
 *    the x and y directions, the columns the incoming and outgoing bond of the
 *    site. The left pattern (-1 1; -1 1) is a local minimum; it becomes the
 *    right pattern (a local maximum, height +2) with probability p; the reverse
 *    (height -2) happens with probability q.
 *  - Schedule: a sweep t is half-sweep s = 0 (sites with (x+y) even) followed
 *    by half-sweep s = 1. Sites of one sublattice share no bond, so the order
 *    inside a half-sweep does not matter.
 *  - Each active site is additionally selected with probability s_sel, so the
 *    effective probabilities are s_sel*p and s_sel*q. This rescales time only:
 *    lambda = 2p/(p+q) - 1 (Sec. I) is unchanged.
 *  - Acceptance uses a k-bit uniform U and integer thresholds P_k, Q_k.
 *  - Heights, Eq. (3): h(x,y) = H0 + sum_{x'<x} sigma_x(x',0)
 *                               + sum_{y'<y} sigma_y(x,y').
 *  - Width, Eq. (4): the second term's prefactor is read as 1/L^2 (the mean
 *    height), which gives W^2 = 1/4 on the striped start as Sec. III states.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11. Round function:     */
/* two 32x32->64 products of counter words 0 and 2 with the multipliers,     */
/* outputs (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped by the Weyl   */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                               uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds. p_eff = s_sel*p, q_eff = s_sel*q. k is the         */
/* smallest k <= k_max with p_eff*2^k and q_eff*2^k both integers; if none,   */
/* k = k_max and P = nearbyint(p_eff*2^k) (round half to even), same for Q.  */
/* A site is accepted iff U < P (minimum) or U < Q (maximum), U uniform on    */
/* [0, 2^k). Returns 0, or -1 for parameters out of range.                    */
/* ------------------------------------------------------------------------ */
ORC_API int orc_thresholds(double p, double q, double s_sel, int k_max,
                           int *k_out, uint64_t *P_out, uint64_t *Q_out)
{
    if (!(p >= 0.0 && p <= 1.0 && q >= 0.0 && q <= 1.0))
        return -1;
    if (!(s_sel > 0.0 && s_sel <= 1.0) || k_max < 1 || k_max > 32)
        return -1;
    double pe = s_sel * p, qe = s_sel * q;
    for (int k = 0; k <= k_max; ++k) {
        double a = ldexp(pe, k), b = ldexp(qe, k);
        if (a == floor(a) && b == floor(b)) {
            *k_out = k;
            *P_out = (uint64_t)a;
            *Q_out = (uint64_t)b;
            return 0;
        }
    }
    int old = fegetround();
    fesetround(FE_TONEAREST);
    double a = nearbyint(ldexp(pe, k_max));
    double b = nearbyint(ldexp(qe, k_max));
    fesetround(old);
    *k_out = k_max;
    *P_out = (uint64_t)a;
    *Q_out = (uint64_t)b;
    return 0;
}

/* 32-bit threshold of the random-sequential variant: nearbyint(p * 2^32). */
ORC_API uint64_t orc_rs_threshold(double p)
{
    int old = fegetround();
    fesetround(FE_TONEAREST);
    double a = nearbyint(ldexp(p, 32));
    fesetround(old);
    return (uint64_t)a;
}

/* ------------------------------------------------------------------------ */
/* Random draws of the checkerboard dynamics.                                 */
/*  site index i = y*L + x; group g = i / 128; word j = (i mod 128) / 32;     */
/*  bit b = i mod 32. Level m of the draw of site (x,y) at sweep t is bit b   */
/*  of word j of Philox4x32-10(ctr = (g mod 2^32, g / 2^32, t, m),            */
/*  key = (seed mod 2^32, seed / 2^32)). U = sum_m bit_m 2^(k-1-m).           */
/* The cache below only remembers the Philox words of the current group; it  */
/* never changes a value.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    uint64_t t;
    int64_t L;
    uint64_t group;
    int levels;
    uint32_t words[32][4];
} draw_cache;

static void draw_cache_init(draw_cache *c, uint64_t seed, uint64_t t, int64_t L)
{
    c->seed = seed;
    c->t = t;
    c->L = L;
    c->group = UINT64_MAX;
    c->levels = 0;
}

static uint64_t site_uniform(draw_cache *c, int64_t x, int64_t y, int k)
{
    uint64_t i = (uint64_t)y * (uint64_t)c->L + (uint64_t)x;
    uint64_t g = i >> 7;
    int j = (int)((i >> 5) & 3u);
    int b = (int)(i & 31u);
    if (g != c->group) {
        c->group = g;
        c->levels = 0;
    }
    uint64_t U = 0;
    for (int m = 0; m < k; ++m) {
        if (m >= c->levels) {
            uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)c->t,
                               (uint32_t)m};
            uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
            orc_philox4x32_10(ctr, key, c->words[m]);
            c->levels = m + 1;
        }
        U = (U << 1) | ((c->words[m][j] >> b) & 1u);
    }
    return U;
}

/* The k-bit uniform of one site, exposed for tests. */
ORC_API uint64_t orc_site_uniform(uint64_t seed, int64_t L, int64_t x, int64_t y,
                                  uint64_t t, int k)
{
    draw_cache c;
    draw_cache_init(&c, seed, t, L);
    return site_uniform(&c, x, y, k);
}

/* ------------------------------------------------------------------------ */
/* Flat ("half filled, striped") start, Sec. III: h(x,y) = (x+y) mod 2, so   */
/* sigma_x(x,y) = +1 iff (x+y) even, and the same for sigma_y. H0 = 0.        */
/* ------------------------------------------------------------------------ */
ORC_API void orc_init_flat(int64_t L, uint8_t *X, uint8_t *Y)
{
    for (int64_t y = 0; y < L; ++y)
        for (int64_t x = 0; x < L; ++x) {
            uint8_t up = ((x + y) % 2 == 0) ? 1 : 0;
            X[y * L + x] = up;
            Y[y * L + x] = up;
        }
}

/* The rule of Eq. (2) at one site: returns +1 (minimum accepted, h += 2),
 * -1 (maximum accepted, h -= 2) or 0, and flips the four bonds on accept. */
static int update_site(int64_t L, uint8_t *X, uint8_t *Y, int64_t x, int64_t y,
                       draw_cache *cache, int k, uint64_t P, uint64_t Q)
{
    int64_t xm = (x == 0) ? L - 1 : x - 1; /* periodic neighbours */
    int64_t ym = (y == 0) ? L - 1 : y - 1;
    uint8_t *left = &X[y * L + xm];  /* sigma_x(x-1,y): bond into the site   */
    uint8_t *right = &X[y * L + x];  /* sigma_x(x,y):   bond out of the site */
    uint8_t *down = &Y[ym * L + x];  /* sigma_y(x,y-1)                       */
    uint8_t *up = &Y[y * L + x];     /* sigma_y(x,y)                         */
    int is_min = (*left == 0) && (*right == 1) && (*down == 0) && (*up == 1);
    int is_max = (*left == 1) && (*right == 0) && (*down == 1) && (*up == 0);
    if (!is_min && !is_max)
        return 0;
    uint64_t U = site_uniform(cache, x, y, k);
    int accept = is_min ? (U < P) : (U < Q);
    if (!accept)
        return 0;
    *left ^= 1;
    *right ^= 1;
    *down ^= 1;
    *up ^= 1;
    return is_min ? 1 : -1;
}

/* One half-sweep s of sweep t: every site with (x+y) mod 2 == s, row-major.
 * Rows may run on several threads: a site only touches its own four bonds,
 * and no bond belongs to two sites of one sublattice. */
static void halfsweep_rows(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                           uint64_t seed, uint64_t t, int s, int k, uint64_t P,
                           uint64_t Q, int threaded)
{
    int64_t dH = 0;
#pragma omp parallel for schedule(static) reduction(+ : dH) if (threaded)
    for (int64_t y = 0; y < L; ++y) {
        draw_cache cache;
        draw_cache_init(&cache, seed, t, L);
        for (int64_t x = (s + y) % 2; x < L; x += 2) {
            int d = update_site(L, X, Y, x, y, &cache, k, P, Q);
            if (d != 0 && x == 0 && y == 0)
                dH += 2 * d;
        }
    }
    *H0 += dH;
}

ORC_API void orc_halfsweep(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                           uint64_t seed, uint64_t t, int s, int k, uint64_t P,
                           uint64_t Q)
{
    halfsweep_rows(L, X, Y, H0, seed, t, s, k, P, Q, L >= 64);
}

/* The same half-sweep, visiting the active sites in a caller-given order
 * (site indices y*L + x). Used to show that the order does not matter. */
ORC_API int orc_halfsweep_ordered(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                                  uint64_t seed, uint64_t t, int s, int k,
                                  uint64_t P, uint64_t Q, const int64_t *order,
                                  int64_t n_order)
{
    draw_cache cache;
    draw_cache_init(&cache, seed, t, L);
    for (int64_t n = 0; n < n_order; ++n) {
        int64_t x = order[n] % L, y = order[n] / L;
        if ((x + y) % 2 != s)
            return -1;
        int d = update_site(L, X, Y, x, y, &cache, k, P, Q);
        if (d != 0 && x == 0 && y == 0)
            *H0 += 2 * d;
    }
    return 0;
}

/* n sweeps starting at sweep index t0. */
ORC_API void orc_sweeps(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                        uint64_t seed, uint64_t t0, int64_t n, int k, uint64_t P,
                        uint64_t Q)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_halfsweep(L, X, Y, H0, seed, t0 + (uint64_t)i, 0, k, P, Q);
        orc_halfsweep(L, X, Y, H0, seed, t0 + (uint64_t)i, 1, k, P, Q);
    }
}

/* n sweeps on a lattice of at most 32 sites, recording the state after every
 * thin-th sweep as a code: bond bit i of X in bit i, bond bit i of Y in bit
 * L*L + i (i = y*L + x). Used by the exact-chain check on a 4x4 lattice. */
ORC_API int orc_sweeps_record(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                              uint64_t seed, uint64_t t0, int64_t n, int k,
                              uint64_t P, uint64_t Q, int64_t thin, uint64_t *codes)
{
    if (L * L > 32 || thin < 1)
        return -1;
    int64_t n_rec = 0;
    for (int64_t i = 0; i < n; ++i) {
        halfsweep_rows(L, X, Y, H0, seed, t0 + (uint64_t)i, 0, k, P, Q, 0);
        halfsweep_rows(L, X, Y, H0, seed, t0 + (uint64_t)i, 1, k, P, Q, 0);
        if ((i + 1) % thin == 0) {
            uint64_t code = 0;
            for (int64_t b = 0; b < L * L; ++b) {
                code |= (uint64_t)X[b] << b;
                code |= (uint64_t)Y[b] << (L * L + b);
            }
            codes[n_rec++] = code;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Random-sequential variant: the paper's own dynamics (Sec. II, random      */
/* update attempts). Sweep t = N = L*L attempts a = 0..N-1, each applied at  */
/* once. Attempt a draws Philox4x32-10(ctr = (a mod 2^32, a / 2^32, t, 256), */
/* key = seed) = (r0, r1, r2, r3): x = (r0*L) >> 32, y = (r1*L) >> 32, and   */
/* the attempt is accepted iff r2 < P32 (minimum) or r2 < Q32 (maximum).     */
/* ------------------------------------------------------------------------ */
ORC_API void orc_rs_sweeps(int64_t L, uint8_t *X, uint8_t *Y, int64_t *H0,
                           uint64_t seed, uint64_t t0, int64_t n, uint64_t P32,
                           uint64_t Q32)
{
    uint64_t N = (uint64_t)L * (uint64_t)L;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        uint64_t t = t0 + (uint64_t)i;
        for (uint64_t a = 0; a < N; ++a) {
            uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), (uint32_t)t, 256u};
            uint32_t r[4];
            orc_philox4x32_10(ctr, key, r);
            int64_t x = (int64_t)(((uint64_t)r[0] * (uint64_t)L) >> 32);
            int64_t y = (int64_t)(((uint64_t)r[1] * (uint64_t)L) >> 32);
            int64_t xm = (x + L - 1) % L, ym = (y + L - 1) % L;
            uint8_t *left = &X[y * L + xm], *right = &X[y * L + x];
            uint8_t *down = &Y[ym * L + x], *up = &Y[y * L + x];
            int is_min = (*left == 0) && (*right == 1) && (*down == 0) && (*up == 1);
            int is_max = (*left == 1) && (*right == 0) && (*down == 1) && (*up == 0);
            int accept = (is_min && r[2] < P32) || (is_max && r[2] < Q32);
            if (!accept)
                continue;
            *left ^= 1;
            *right ^= 1;
            *down ^= 1;
            *up ^= 1;
            if (x == 0 && y == 0)
                *H0 += is_min ? 2 : -2;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Domain-decomposed random-sequential dynamics (Sec. II: blocks with dead   */
/* borders, the origin moved at random every MCS, random update attempts     */
/* inside each block). Sweep t:                                               */
/*  - offsets (ox, oy) = (r0 mod C, r1 mod C) of Philox(ctr = (0, 0, t, 768)); */
/*  - cell (i, j), i, j < L/C, has origin ((ox + iC) mod L, (oy + jC) mod L)  */
/*    and id c = j*(L/C) + i;                                                 */
/*  - it receives C*C attempts a = 0, 1, ... in order; attempt a uses words   */
/*    (r0, r1) (a even) or (r2, r3) (a odd) of Philox(ctr = (c, a/2, t,       */
/*    1024)): local x = first & (C-1), local y = (first >> 16) & (C-1),       */
/*    u = second. Attempts on the cell's dead border (local x = 0 or local   */
/*    y = 0) do nothing; elsewhere a minimum moves iff u < P32, a maximum iff */
/*    u < Q32 (32-bit thresholds, no selection factor).                       */
/* Two dead edges suffice, as in the paper's Fig. 1: a site's move flips its */
/* four bonds, and the only bonds a cell shares with its neighbours in x and  */
/* y join its last column (row) to their dead first column (row). Cells thus  */
/* share no bond that anyone flips, and the cell order does not matter. C    */
/* must be a power of two dividing L.                                         */
/* ------------------------------------------------------------------------ */
ORC_API int orc_ddrs_sweeps(int64_t L, int64_t C, uint8_t *X, uint8_t *Y, int64_t *H0,
                            uint64_t seed, uint64_t t0, int64_t n, uint64_t P32,
                            uint64_t Q32)
{
    if (C < 4 || (C & (C - 1)) != 0 || L % C != 0)
        return -1;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t ncell = L / C;
    for (int64_t it = 0; it < n; ++it) {
        uint64_t t = t0 + (uint64_t)it;
        uint32_t octr[4] = {0, 0, (uint32_t)t, 768u}, o[4];
        orc_philox4x32_10(octr, key, o);
        int64_t ox = (int64_t)(o[0] & (uint32_t)(C - 1));
        int64_t oy = (int64_t)(o[1] & (uint32_t)(C - 1));
        for (int64_t cj = 0; cj < ncell; ++cj)
            for (int64_t ci = 0; ci < ncell; ++ci) {
                uint64_t c = (uint64_t)(cj * ncell + ci);
                int64_t x0 = (ox + ci * C) % L, y0 = (oy + cj * C) % L;
                uint32_t r[4] = {0, 0, 0, 0};
                for (int64_t a = 0; a < C * C; ++a) {
                    if (a % 2 == 0) {
                        uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(a / 2), (uint32_t)t, 1024u};
                        orc_philox4x32_10(ctr, key, r);
                    }
                    uint32_t first = (a % 2 == 0) ? r[0] : r[2];
                    uint32_t u = (a % 2 == 0) ? r[1] : r[3];
                    int64_t lx = (int64_t)(first & (uint32_t)(C - 1));
                    int64_t ly = (int64_t)((first >> 16) & (uint32_t)(C - 1));
                    if (lx == 0 || ly == 0)
                        continue;
                    int64_t x = (x0 + lx) % L, y = (y0 + ly) % L;
                    int64_t xm = (x == 0) ? L - 1 : x - 1, ym = (y == 0) ? L - 1 : y - 1;
                    uint8_t *left = &X[y * L + xm], *right = &X[y * L + x];
                    uint8_t *down = &Y[ym * L + x], *up = &Y[y * L + x];
                    int is_min = (*left == 0) && (*right == 1) && (*down == 0) && (*up == 1);
                    int is_max = (*left == 1) && (*right == 0) && (*down == 1) && (*up == 0);
                    int accept = (is_min && u < P32) || (is_max && u < Q32);
                    if (!accept)
                        continue;
                    *left ^= 1;
                    *right ^= 1;
                    *down ^= 1;
                    *up ^= 1;
                    if (x == 0 && y == 0)
                        *H0 += is_min ? 2 : -2;
                }
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* A window of a larger periodic L x L lattice, for checking very large runs  */
/* site by site. The window holds the bonds of the sites                     */
/*   (x0 + i mod L, y0 + j mod L),  0 <= i < w, 0 <= j < h,                   */
/* as WX[j*w + i], WY[j*w + i]. Random draws, sublattices and sweep indices   */
/* use the global coordinates, so inside the window the dynamics is the full  */
/* lattice's. Sites with i = 0 or j = 0 are never updated (a bond they need    */
/* lies outside) and nothing outside is simulated, so errors enter from the   */
/* edges and move inward by at most one site per half-sweep: after n sweeps   */
/* sites farther than 2n + 1 from every edge are exact.                       */
/* ------------------------------------------------------------------------ */
ORC_API void orc_window_init_flat(int64_t x0, int64_t y0, int64_t w, int64_t h,
                                  uint8_t *WX, uint8_t *WY)
{
    for (int64_t j = 0; j < h; ++j)
        for (int64_t i = 0; i < w; ++i) {
            uint8_t up = ((x0 + i + y0 + j) % 2 == 0) ? 1 : 0; /* L even */
            WX[j * w + i] = up;
            WY[j * w + i] = up;
        }
}

ORC_API void orc_window_sweeps(int64_t L, int64_t x0, int64_t y0, int64_t w, int64_t h,
                               uint8_t *WX, uint8_t *WY, uint64_t seed, uint64_t t0,
                               int64_t n, int k, uint64_t P, uint64_t Q)
{
    for (int64_t it = 0; it < n; ++it) {
        uint64_t t = t0 + (uint64_t)it;
        for (int s = 0; s < 2; ++s) {
            /* rows of one half-sweep touch disjoint bonds (as in halfsweep_rows) */
#pragma omp parallel for schedule(static) if (w * h >= 4096)
            for (int64_t j = 1; j < h; ++j) {
                draw_cache cache;
                draw_cache_init(&cache, seed, t, L);
                for (int64_t i = 1; i < w; ++i) {
                    int64_t gx = (x0 + i) % L, gy = (y0 + j) % L;
                    if ((gx + gy) % 2 != s)
                        continue;
                    uint8_t *left = &WX[j * w + i - 1], *right = &WX[j * w + i];
                    uint8_t *down = &WY[(j - 1) * w + i], *up = &WY[j * w + i];
                    int is_min = (*left == 0) && (*right == 1) && (*down == 0) && (*up == 1);
                    int is_max = (*left == 1) && (*right == 0) && (*down == 1) && (*up == 0);
                    if (!is_min && !is_max)
                        continue;
                    uint64_t U = site_uniform(&cache, gx, gy, k);
                    if (is_min ? (U < P) : (U < Q)) {
                        *left ^= 1;
                        *right ^= 1;
                        *down ^= 1;
                        *up ^= 1;
                    }
                }
            }
        }
    }
}

/* Height of one site straight from packed bit-planes (the C-ABI layout: L
 * rows of L/32 little-endian 32-bit words per plane, bit b of word w = bond
 * at x = 32w + b), following Eq. (3): along row 0, then up column x. */
static int packed_bit(const uint32_t *plane, int64_t L, int64_t x, int64_t y)
{
    return (int)((plane[y * (L / 32) + x / 32] >> (x % 32)) & 1u);
}

ORC_API int64_t orc_height_packed(int64_t L, const uint32_t *Xw, const uint32_t *Yw,
                                  int64_t H0, int64_t x, int64_t y)
{
    int64_t h = H0;
    for (int64_t xp = 0; xp < x; ++xp)
        h += 2 * packed_bit(Xw, L, xp, 0) - 1;
    for (int64_t yp = 0; yp < y; ++yp)
        h += 2 * packed_bit(Yw, L, x, yp) - 1;
    return h;
}

/* ------------------------------------------------------------------------ */
/* Heights, Eq. (3), with sigma = 2*bit - 1 and 0-based sums:                 */
/*   h(x,0) = H0 + sum_{x'<x} sigma_x(x',0)                                   */
/*   h(x,y) = h(x,0) + sum_{y'<y} sigma_y(x,y')                               */
/* ------------------------------------------------------------------------ */
ORC_API void orc_heights(int64_t L, const uint8_t *X, const uint8_t *Y, int64_t H0,
                         int64_t *h)
{
    int64_t acc = H0;
    for (int64_t x = 0; x < L; ++x) {
        h[x] = acc;
        acc += 2 * (int64_t)X[x] - 1;
    }
    for (int64_t y = 1; y < L; ++y)
        for (int64_t x = 0; x < L; ++x)
            h[y * L + x] = h[(y - 1) * L + x] + 2 * (int64_t)Y[(y - 1) * L + x] - 1;
}

static void put_i128(i128 v, int64_t out[2])
{
    out[0] = (int64_t)(uint64_t)((unsigned __int128)v);          /* low 64 bits  */
    out[1] = (int64_t)(uint64_t)(((unsigned __int128)v) >> 64);  /* high 64 bits */
}

/* Exact power sums of the heights: out[2*(n-1)], out[2*(n-1)+1] = low and
 * high 64-bit halves of S_n = sum (h - c)^n, n = 1..4, as 128-bit integers. */
ORC_API void orc_power_sums(int64_t L, const int64_t *h, int64_t c, int64_t out[8])
{
    i128 s[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < L * L; ++i) {
        i128 d = (i128)(h[i] - c);
        i128 dn = d;
        for (int n = 0; n < 4; ++n) {
            s[n] += dn;
            dn *= d;
        }
    }
    for (int n = 0; n < 4; ++n)
        put_i128(s[n], &out[2 * n]);
}

/* W^2 of Eq. (4) with the 1/L^2 reading:
 *   W^2 = (1/N) sum h^2 - ((1/N) sum h)^2 = (N*S2 - S1^2) / N^2, N = L*L,
 * with the numerator formed exactly in 128-bit integers from sums about c
 * (the numerator does not depend on c), then rounded once to double and
 * divided by double(N)*double(N). */
ORC_API double orc_width2(int64_t L, const int64_t *h, int64_t c)
{
    i128 s1 = 0, s2 = 0;
    for (int64_t i = 0; i < L * L; ++i) {
        i128 d = (i128)(h[i] - c);
        s1 += d;
        s2 += d * d;
    }
    i128 N = (i128)L * (i128)L;
    i128 num = N * s2 - s1 * s1;
    return (double)num / ((double)N * (double)N);
}

/* Skewness and excess kurtosis of the heights from the exact sums about c:
 *   mu = S1/N, m2 = S2/N - mu^2, m3 = S3/N - 3 mu S2/N + 2 mu^3,
 *   m4 = S4/N - 4 mu S3/N + 6 mu^2 S2/N - 3 mu^4,
 *   skew = m3 / m2^(3/2), kurt = m4 / m2^2 - 3,
 * evaluated in long double. out = {skew, kurt}. */
ORC_API void orc_skew_kurt(int64_t L, const int64_t *h, int64_t c, double out[2])
{
    int64_t raw[8];
    orc_power_sums(L, h, c, raw);
    long double S[4];
    for (int n = 0; n < 4; ++n) {
        i128 v = (i128)(((unsigned __int128)(uint64_t)raw[2 * n + 1] << 64) |
                        (unsigned __int128)(uint64_t)raw[2 * n]);
        S[n] = (long double)v;
    }
    long double N = (long double)L * (long double)L;
    long double mu = S[0] / N;
    long double a2 = S[1] / N, a3 = S[2] / N, a4 = S[3] / N;
    long double m2 = a2 - mu * mu;
    long double m3 = a3 - 3.0L * mu * a2 + 2.0L * mu * mu * mu;
    long double m4 = a4 - 4.0L * mu * a3 + 6.0L * mu * mu * a2 - 3.0L * mu * mu * mu * mu;
    out[0] = (double)(m3 / powl(m2, 1.5L));
    out[1] = (double)(m4 / (m2 * m2) - 3.0L);
}

/* ------------------------------------------------------------------------ */
/* Sampling times. Sec. III grows the gap between measurements             */
/* exponentially; here the n sample times are log-spaced over [1, T]:       */
/*   t_j = max(round(T^(j/(n-1))), t_{j-1} + 1), j = 0..n-1, t_{n-1} = T,   */
/* preceded by the t = 0 record. out must hold n + 1 entries. Returns 0, or  */
/* -1 when n < 2 or n > T.                                                   */
/* ------------------------------------------------------------------------ */
ORC_API int orc_sample_times(uint64_t T, int n, uint64_t *out)
{
    if (n < 2 || (uint64_t)n > T)
        return -1;
    out[0] = 0;
    uint64_t prev = 0;
    for (int j = 0; j < n; ++j) {
        uint64_t v = (uint64_t)llround(pow((double)T, (double)j / (double)(n - 1)));
        if (v <= prev)
            v = prev + 1;
        out[j + 1] = v;
        prev = v;
    }
    if (out[n] != T)
        return -1;
    return 0;
}
