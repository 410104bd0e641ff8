/*
 * gbmc_oracle.c -- plain, slow CPU oracle for checkerboard Metropolis sweeps of
 * Ising-type lattices and population annealing (Weigel, "Monte Carlo methods for
 * massively parallel computers", arXiv:1709.04394).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load or call this code. It shares no code, header,
 * table or constant with the CUDA library and includes nothing from it.
 *
 * Every routine follows the paper's steps in the paper's order, one site (or
 * one replica) at a time, with no blocking, fusion or reordering:
 *   - Ising Hamiltonian, Eq. (7), with h_i = 0 and periodic boundaries (Sec. 3).
 *   - Single-spin-flip Metropolis rule, the four-step list of Sec. 3.1 and
 *     Eq. (8): flip if dE <= 0 or r < exp(-beta dE), r uniform in [0,1).
 *   - Checkerboard order: the even sub-lattice, then the odd one (Sec. 3.1,
 *     Fig. 5; the offset 0 / offset 1 kernel calls described there).
 *   - Philox4x32-10 counter-based generator: the mulhi/mullo round of Sec. 4
 *     with the constants of Salmon et al. (2011), ten rounds.
 *   - Population annealing, the five-step algorithm of Sec. 5.4 with the
 *     normaliser Q_i of Eq. (13).
 *   - Bimodal +-J couplings of the Edwards-Anderson spin glass (Sec. 6).
 *
 * Readings where the paper is silent (all of them are conventions shared with
 * the CUDA path only through their written definition):
 *   R1 key = (seed lo, seed hi); Metropolis counter = (q, t, r, c3) with
 *      k = rank of the site among colour-c sites in row-major order, q = k>>2,
 *      word k&3; t = global sweep counter; r = replica slot;
 *      c3 = purpose<<28 | colour<<27 | instance.
 *      Purposes: METRO 0, INIT 1 (q = site>>2, word site&3, t = 0),
 *      RESAMPLE 2 (draw k: q = k>>1, t = step, r = 0, 64-bit word k&1),
 *      COUPLING 3 (bond b = 3 site + mu: q = b>>2, word b&3, t = r = 0).
 *   R2 r = u 2^-32 with u the 32-bit word, so "r < p" is "u <= ceil(p 2^32) - 1".
 *   R3 dE = 0 is accepted (the rule says dE <= 0).
 *   R4 colour(x,y[,z]) = (x+y[+z]) mod 2; colour 0 first.
 *   R5 PA step order: resample to beta_i, theta sweeps at beta_i, measure.
 *   R6 constant population R, multinomial resampling with integer weights
 *      W(E) = floor(2^s exp(-dbeta (E - Emin))), s = 63 - ceil(log2 R); the
 *      cumulative sums C_j are taken in replica order; draw k picks the least
 *      j with C_j > floor(U64_k C_R / 2^64); children of parent j are placed
 *      contiguously, parents in increasing order.
 *   R7 ln Q_i = -dbeta Emin + ln sum_E h(E) exp(-dbeta (E - Emin)) - ln R,
 *      summed over energy levels in increasing E.
 *   R9 J_{i,mu} = +1 if the top bit of its COUPLING word is 0, else -1.
 *  R10 ln Z(beta_0 = 0) = N ln 2; ln Z_i = ln Z_{i-1} + ln Q_i.
 *  R16 double checkerboard: see orc_dcb_sweeps.
 *  R17 nearest-integer resampling, variable population: see
 *      orc_resample_nearest.
 *  R19 Swendsen-Wang (Sec. 3.3): see orc_sw_update.
 *  R20 Poisson resampling: see orc_exp_neg, orc_poisson, orc_resample_poisson.
 *  R18 multi-spin coding across replicas (Sec. 5.4): replicas 32 w .. 32 w +
 *      31 share, at each site and visit, one Philox word (purpose MSC 5,
 *      counter (k >> 2, t, w, c3), word k & 3) that seeds an LCG; replica
 *      32 w + b compares the LCG's (b + 1)-th output with the threshold.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PURPOSE_METRO 0u
#define ORC_PURPOSE_INIT 1u
#define ORC_PURPOSE_RESAMPLE 2u
#define ORC_PURPOSE_COUPLING 3u
#define ORC_PURPOSE_MSC 5u
#define ORC_PURPOSE_SW_BOND 6u
#define ORC_PURPOSE_SW_FLIP 7u

/* The linear congruential generator of the multi-spin-coded sweeps (reading
 * R18): x -> a x + c mod 2^32 with the constants of Numerical Recipes. */
#define ORC_LCG_A 1664525u
#define ORC_LCG_C 1013904223u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Sec. 4, counter-based generators).                         */
/* One round: the two 64-bit products R*M give L' = mullo and                 */
/* R' = mulhi xor key xor L for the two word pairs, with the pair            */
/* permutation of the 4x32 variant; the key is advanced by the Weyl           */
/* increments between rounds.                                                 */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t orc_word(uint64_t seed, uint32_t q, uint32_t t, uint32_t r, uint32_t c3,
                         unsigned lane)
{
    uint32_t ctr[4] = {q, t, r, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[lane & 3u];
}

static uint32_t orc_c3(uint32_t purpose, uint32_t colour, uint32_t instance)
{
    return (purpose << 28) | (colour << 27) | instance;
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: N = L^dim sites, x fastest, periodic boundaries.        */
/* ------------------------------------------------------------------------ */
static int64_t orc_nsites(int dim, int L)
{
    int64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= L;
    return n;
}

static void orc_coords(int dim, int L, int64_t site, int *x, int *y, int *z)
{
    *x = (int)(site % L);
    *y = (int)((site / L) % L);
    *z = dim == 3 ? (int)(site / ((int64_t)L * L)) : 0;
}

static int64_t orc_site(int dim, int L, int x, int y, int z)
{
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    z = ((z % L) + L) % L;
    return dim == 3 ? ((int64_t)z * L + y) * L + x : (int64_t)y * L + x;
}

/* Neighbour n (0..2*dim-1) of a site: even n = forward along axis n/2, odd n =
 * backward. The coupling of that bond, J_{i,mu} of the forward bond leaving
 * site i along mu (stored as J[3*i+mu] for dim 3; all +1 when J == NULL). */
static int64_t orc_neighbour(int dim, int L, int64_t site, int n, const int8_t *J, int *Jn)
{
    int x, y, z;
    orc_coords(dim, L, site, &x, &y, &z);
    int axis = n / 2, fwd = (n % 2) == 0;
    int dx = axis == 0 ? 1 : 0, dy = axis == 1 ? 1 : 0, dz = axis == 2 ? 1 : 0;
    int64_t nb;
    if (fwd) {
        nb = orc_site(dim, L, x + dx, y + dy, z + dz);
        *Jn = J ? J[3 * site + axis] : 1;
    } else {
        nb = orc_site(dim, L, x - dx, y - dy, z - dz);
        *Jn = J ? J[3 * nb + axis] : 1;
    }
    return nb;
}

/* ------------------------------------------------------------------------ */
/* Thresholds (reading R2): T(dE) = ceil(exp(-beta dE) 2^32) - 1, so that a   */
/* 32-bit word u satisfies u 2^-32 < exp(-beta dE)  <=>  u <= T(dE).          */
/* out[m] = T(4(m+1)) for m = 0 .. ndE-1.                                     */
/* ------------------------------------------------------------------------ */
void orc_thresholds(double beta, int ndE, int64_t *out)
{
    for (int m = 0; m < ndE; ++m) {
        double dE = 4.0 * (double)(m + 1);
        double p = exp(-(beta * dE));
        double scaled = ldexp(p, 32);
        out[m] = (int64_t)ceil(scaled) - 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Step 1 of the Sec. 3.1 list: initial configuration (all up, or uniformly   */
/* random from the INIT purpose: s = +1 if the word's top bit is 0).          */
/* ------------------------------------------------------------------------ */
void orc_init_spins(int dim, int L, uint64_t seed, uint32_t instance, uint32_t replica,
                    int random_start, int8_t *s)
{
    int64_t N = orc_nsites(dim, L);
    for (int64_t i = 0; i < N; ++i) {
        if (!random_start) {
            s[i] = 1;
        } else {
            uint32_t u = orc_word(seed, (uint32_t)(i >> 2), 0u, replica,
                                  orc_c3(ORC_PURPOSE_INIT, 0u, instance), (unsigned)(i & 3));
            s[i] = (u >> 31) ? -1 : 1;
        }
    }
}

/* Bimodal couplings P(J = +1) = P(J = -1) = 1/2 (Sec. 6), three forward bonds
 * per site of a dim-3 lattice, J[3*site + mu]. */
void orc_couplings(int L, uint64_t seed, uint32_t instance, int8_t *J)
{
    int64_t N = orc_nsites(3, L);
    for (int64_t i = 0; i < N; ++i) {
        for (int mu = 0; mu < 3; ++mu) {
            int64_t b = 3 * i + mu;
            uint32_t u = orc_word(seed, (uint32_t)(b >> 2), 0u, 0u,
                                  orc_c3(ORC_PURPOSE_COUPLING, 0u, instance), (unsigned)(b & 3));
            J[b] = (u >> 31) ? -1 : 1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Steps 2-3 of the Sec. 3.1 list for every site of one sub-lattice.          */
/* ------------------------------------------------------------------------ */
/* Metropolis updates of the colour-`colour` sites; with tile > 0 (2D only)
 * just those in tiles of coarse colour `coarse` (Fig. 5, right: tile (a, b)
 * holds the sites with x / tile = a, y / tile = b; its coarse colour is
 * (a + b) mod 2). The updated sites are never neighbours, so the order within
 * the loop does not matter. */
/* Uniform of replica `replica` at colour-rank k in the multi-spin-coded
 * sweeps (reading R18): the Philox word of (q = k >> 2, t, group = replica /
 * 32, purpose MSC) seeds the LCG, whose (replica mod 32) + 1-th output it is. */
static uint32_t orc_msc_uniform(uint64_t seed, uint64_t k, uint32_t t, uint32_t replica, int colour,
                                uint32_t instance)
{
    uint32_t x = orc_word(seed, (uint32_t)(k >> 2), t, replica >> 5,
                          orc_c3(ORC_PURPOSE_MSC, (uint32_t)colour, instance), (unsigned)(k & 3));
    for (uint32_t j = 0; j <= (replica & 31u); ++j) x = ORC_LCG_A * x + ORC_LCG_C;
    return x;
}

static void orc_update_sites(int dim, int L, int8_t *s, const int8_t *J, const int64_t *thr,
                             uint64_t seed, uint32_t instance, uint32_t replica, uint32_t t, int colour,
                             int tile, int coarse, int msc)
{
    int64_t N = orc_nsites(dim, L);
    uint32_t c3 = orc_c3(ORC_PURPOSE_METRO, (uint32_t)colour, instance);
    for (int64_t i = 0; i < N; ++i) {
        int x, y, z;
        orc_coords(dim, L, i, &x, &y, &z);
        if (((x + y + z) & 1) != colour) continue;
        if (tile > 0 && ((x / tile + y / tile) & 1) != coarse) continue;
        /* rank among the sites of this colour, row-major */
        int64_t row = dim == 3 ? (int64_t)z * L + y : (int64_t)y;
        int64_t k = row * (L / 2) + (x >> 1);
        /* dE_k = 2 s_k sum_nn J s_j */
        int h = 0;
        for (int n = 0; n < 2 * dim; ++n) {
            int Jn;
            int64_t nb = orc_neighbour(dim, L, i, n, J, &Jn);
            h += Jn * s[nb];
        }
        int dE = 2 * s[i] * h;
        int accept;
        if (dE <= 0) {
            accept = 1;
        } else {
            uint32_t u = msc ? orc_msc_uniform(seed, (uint64_t)k, t, replica, colour, instance)
                             : orc_word(seed, (uint32_t)(k >> 2), t, replica, c3, (unsigned)(k & 3));
            accept = (int64_t)u <= thr[dE / 4 - 1];
        }
        if (accept) s[i] = (int8_t)(-s[i]);
    }
}

void orc_halfsweep(int dim, int L, int8_t *s, const int8_t *J, const int64_t *thr,
                   uint64_t seed, uint32_t instance, uint32_t replica, uint32_t t, int colour)
{
    orc_update_sites(dim, L, s, J, thr, seed, instance, replica, t, colour, 0, 0, 0);
}

/* The 32 uniforms of one multi-spin-coded group at colour-rank k (tests). */
void orc_msc_uniforms(uint64_t seed, uint64_t k, uint32_t t, uint32_t group, int colour, uint32_t instance,
                      uint32_t *out)
{
    for (uint32_t b = 0; b < 32; ++b) out[b] = orc_msc_uniform(seed, k, t, 32u * group + b, colour, instance);
}

/* n checkerboard sweeps with the multi-spin-coded random numbers (reading
 * R18) of replica `replica`: the same Metropolis rule and order as
 * orc_sweeps, only the uniform of each (site, visit) differs. */
void orc_msc_sweeps(int dim, int L, int8_t *s, const int8_t *J, double beta, uint64_t seed,
                    uint32_t instance, uint32_t replica, uint32_t t0, uint32_t n)
{
    int64_t thr[3];
    orc_thresholds(beta, dim, thr);
    for (uint32_t m = 0; m < n; ++m)
        for (int colour = 0; colour < 2; ++colour)
            orc_update_sites(dim, L, s, J, thr, seed, instance, replica, t0 + m, colour, 0, 0, 1);
}

/* Double checkerboard with k hits per tile (Sec. 3.1, Fig. 5 right, the
 * multi-hit variant): n_rounds rounds of the 2D lattice cut into tile x tile
 * tiles (L a multiple of 2 tile). A round takes the tiles of coarse colour 0,
 * then those of coarse colour 1; the tiles of one coarse colour each get k
 * full checkerboard sweeps (fine colour 0, then 1) while every site outside
 * them stays fixed. Reading R16: the j-th sweep of a tile in round m uses the
 * sweep counter t0 + k m + j for the Philox words of its sites, so every site
 * is visited once per counter value, as in the plain sweeps. */
void orc_dcb_sweeps(int L, int tile, int8_t *s, double beta, uint64_t seed, uint32_t instance,
                    uint32_t replica, uint32_t t0, uint32_t k, uint32_t n_rounds)
{
    int64_t thr[3];
    orc_thresholds(beta, 2, thr);
    for (uint32_t m = 0; m < n_rounds; ++m)
        for (int coarse = 0; coarse < 2; ++coarse)
            for (uint32_t j = 0; j < k; ++j)
                for (int colour = 0; colour < 2; ++colour)
                    orc_update_sites(2, L, s, NULL, thr, seed, instance, replica, t0 + k * m + j, colour,
                                     tile, coarse, 0);
}

/* n full sweeps (even sub-lattice, then odd), sweep counters t0 .. t0+n-1. */
void orc_sweeps(int dim, int L, int8_t *s, const int8_t *J, double beta, uint64_t seed,
                uint32_t instance, uint32_t replica, uint32_t t0, uint32_t n)
{
    int64_t thr[3];
    orc_thresholds(beta, dim, thr);
    for (uint32_t m = 0; m < n; ++m) {
        orc_halfsweep(dim, L, s, J, thr, seed, instance, replica, t0 + m, 0);
        orc_halfsweep(dim, L, s, J, thr, seed, instance, replica, t0 + m, 1);
    }
}

/* Eq. (7): E = -sum_<ij> J_ij s_i s_j over the forward bonds; M = sum_i s_i. */
void orc_observables(int dim, int L, const int8_t *s, const int8_t *J, int64_t *E, int64_t *M)
{
    int64_t N = orc_nsites(dim, L);
    int64_t e = 0, m = 0;
    for (int64_t i = 0; i < N; ++i) {
        for (int axis = 0; axis < dim; ++axis) {
            int Jn;
            int64_t nb = orc_neighbour(dim, L, i, 2 * axis, J, &Jn);
            e -= (int64_t)Jn * s[i] * s[nb];
        }
        m += s[i];
    }
    *E = e;
    *M = m;
}

/* ------------------------------------------------------------------------ */
/* Sec. 5.4, step 2: resampling from beta_{i-1} to beta_i = beta_{i-1}+dbeta. */
/* E[R]: the replicas' energies. Writes counts[R] (number of copies of each   */
/* replica) and returns ln Q_i (Eq. (13), reading R7). Readings R6, R1.      */
/* ------------------------------------------------------------------------ */
static int orc_cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int orc_ceil_log2(uint64_t R)
{
    int b = 0;
    while (((uint64_t)1 << b) < R) ++b;
    return b;
}

/* ln Q_i of Eq. (13) for the R replicas' energies E (reading R7), and E_min. */
static double orc_lnQ(uint32_t R, const int64_t *E, double dbeta, int64_t *Emin_out)
{
    /* minimum energy of the population */
    int64_t Emin = E[0];
    for (uint32_t j = 1; j < R; ++j)
        if (E[j] < Emin) Emin = E[j];

    /* ln Q_i over energy levels in increasing order: copy, sort, run-length */
    int64_t *sorted = (int64_t *)malloc(sizeof(int64_t) * R);
    memcpy(sorted, E, sizeof(int64_t) * R);
    qsort(sorted, R, sizeof(int64_t), orc_cmp_i64);
    double sum = 0.0;
    uint32_t a = 0;
    while (a < R) {
        uint32_t b = a;
        while (b < R && sorted[b] == sorted[a]) ++b;
        double h = (double)(b - a);
        sum += h * exp(-(dbeta * (double)(sorted[a] - Emin)));
        a = b;
    }
    free(sorted);
    *Emin_out = Emin;
    return -dbeta * (double)Emin + log(sum) - log((double)R);
}

/* The 64-bit uniform of resampling draw k (reading R1: purpose RESAMPLE). */
static uint64_t orc_resample_u64(uint64_t seed, uint32_t instance, uint32_t step, uint32_t k)
{
    uint32_t ctr[4] = {k >> 1, step, 0u, orc_c3(ORC_PURPOSE_RESAMPLE, 0u, instance)};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    unsigned l = k & 1u;
    return ((uint64_t)out[2 * l + 1] << 32) | (uint64_t)out[2 * l];
}

double orc_resample(uint32_t R, const int64_t *E, double dbeta, uint64_t seed,
                    uint32_t instance, uint32_t step, uint32_t *counts)
{
    int64_t Emin;
    double lnQ = orc_lnQ(R, E, dbeta, &Emin);

    /* integer weights and their cumulative sums in replica order */
    int s = 63 - orc_ceil_log2(R);
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * R);
    uint64_t acc = 0;
    for (uint32_t j = 0; j < R; ++j) {
        double w = exp(-(dbeta * (double)(E[j] - Emin)));
        uint64_t W = (uint64_t)floor(ldexp(w, s));
        acc += W;
        C[j] = acc;
        counts[j] = 0;
    }
    uint64_t total = acc;

    /* R multinomial draws */
    for (uint32_t k = 0; k < R; ++k) {
        uint64_t U = orc_resample_u64(seed, instance, step, k);
        uint64_t x = (uint64_t)(((unsigned __int128)U * (unsigned __int128)total) >> 64);
        /* least j with C_j > x, by bisection over the increasing C */
        uint32_t lo = 0, hi = R - 1;
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (C[mid] > x) hi = mid;
            else lo = mid + 1;
        }
        counts[lo] += 1;
    }
    free(C);
    return lnQ;
}

/* Sec. 5.4 step 2 with nearest-integer resampling and a variable population
 * (reading R17). Replica j (of R_prev) gets tau_j = R0 W_j / C copies in
 * expectation, the weight e^{-dbeta E_j} / Q_i of the paper rescaled by
 * R0 / R_prev so that the expected population is R0 at every step, with
 * integer weights W_j = floor(2^s exp(-dbeta (E_j - Emin))), s = 63 -
 * ceil(log2 cap), and C = sum_j W_j: n_j = floor(tau_j) plus one more copy
 * with probability frac(tau_j), i.e. iff floor(U64_j C / 2^64) < (R0 W_j mod C)
 * (U64_j: resampling word j). Writes counts[R_prev], *R_new = sum_j n_j;
 * returns ln Q_i of Eq. (13) with R_{i-1} = R_prev. */
double orc_resample_nearest(uint32_t R_prev, const int64_t *E, double dbeta, uint32_t R0, uint32_t cap,
                            uint64_t seed, uint32_t instance, uint32_t step, uint32_t *counts,
                            uint64_t *R_new)
{
    int64_t Emin;
    double lnQ = orc_lnQ(R_prev, E, dbeta, &Emin);
    int s = 63 - orc_ceil_log2(cap);
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * R_prev);
    uint64_t C = 0;
    for (uint32_t j = 0; j < R_prev; ++j) {
        W[j] = (uint64_t)floor(ldexp(exp(-(dbeta * (double)(E[j] - Emin))), s));
        C += W[j];
    }
    uint64_t total = 0;
    for (uint32_t j = 0; j < R_prev; ++j) {
        uint64_t num = (uint64_t)R0 * W[j];
        uint64_t n0 = num / C, rem = num % C;
        uint64_t U = orc_resample_u64(seed, instance, step, j);
        uint64_t x = (uint64_t)(((unsigned __int128)U * (unsigned __int128)C) >> 64);
        counts[j] = (uint32_t)(n0 + (x < rem ? 1u : 0u));
        total += counts[j];
    }
    free(W);
    *R_new = total;
    return lnQ;
}

/* e^{-x} for x >= 0 (reading R20) by Cody and Waite's range reduction,
 * x = k ln2 + r with k = floor(x / ln2 + 1/2), |r| <= ln2 / 2, ln2 split into
 * a head whose last 11 mantissa bits are zero (so k * head is exact for the
 * k < 2^11 that occur) and the remainder, then
 * e^{-r} from its Taylor series to degree 20 by Horner's rule, s <- 1 - (r/n) s
 * for n = 20 .. 1, and an exact scaling by 2^-k. Every step is one IEEE fp64
 * operation (this file is compiled without contraction), so any IEEE machine
 * computes the same bits. x > 700 gives 0. */
#define ORC_LN2_HI 0.693147180559890330187045037746429443359375
#define ORC_LN2_LO 5.4979230187083711552420206887059365096458314e-14
double orc_exp_neg(double x)
{
    if (x > 700.0) return 0.0;
    double k = floor(x / 0.6931471805599453094172321 + 0.5);
    double r = (x - k * ORC_LN2_HI) - k * ORC_LN2_LO;
    double s = 1.0;
    for (int n = 20; n >= 1; --n) s = 1.0 - (r / (double)n) * s;
    return ldexp(s, -(int)k);
}

/* Poisson(tau) count by inversion (reading R20): u = the top 53 bits of U64
 * as a fraction; n is the least count with u < F(n), the cumulative Poisson
 * probabilities built term by term (p_0 = e^{-tau}, p_n = p_{n-1} (tau / n));
 * past the mode, a term too small to change F ends the search (u within
 * rounding of 1). Returns UINT32_MAX if tau > 700 (e^{-tau} underflows). */
uint32_t orc_poisson(double tau, uint64_t U64)
{
    if (tau > 700.0) return UINT32_MAX;
    double u = (double)(U64 >> 11) * 0x1.0p-53;
    double p = orc_exp_neg(tau), F = p;
    uint32_t n = 0;
    while (u >= F && n < 100000u) {
        n += 1;
        p = p * (tau / (double)n);
        double Fn = F + p;
        if (Fn == F && (double)n > tau) break; /* the sum has saturated below u */
        F = Fn;
    }
    return n;
}

/* The Poisson(tau) copies of replica j (reading R20): tau <= 500 from its
 * resampling word; a larger tau as the sum of m = ceil(tau / 500) independent
 * Poisson(tau / m) counts, piece p drawn from the resampling word of the same
 * replica with counter field r = p (the plain word is p = 0). */
static uint32_t orc_poisson_copies(double tau, uint64_t seed, uint32_t instance, uint32_t step, uint32_t j)
{
    if (tau <= 500.0) return orc_poisson(tau, orc_resample_u64(seed, instance, step, j));
    uint32_t m = (uint32_t)ceil(tau / 500.0);
    double part = tau / (double)m;
    uint32_t n = 0;
    for (uint32_t p = 0; p < m; ++p) {
        uint32_t ctr[4] = {j >> 1, step, p, orc_c3(ORC_PURPOSE_RESAMPLE, 0u, instance)};
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        unsigned l = j & 1u;
        n += orc_poisson(part, ((uint64_t)out[2 * l + 1] << 32) | (uint64_t)out[2 * l]);
    }
    return n;
}

/* Sec. 5.4 step 2 with Poisson resampling and a variable population (reading
 * R20): replica j gets Poisson(tau_j) copies, tau_j = R0 W_j / C as in
 * orc_resample_nearest (in fp64: the rounded product R0 W_j and sum C).
 * Returns ln Q_i. */
double orc_resample_poisson(uint32_t R_prev, const int64_t *E, double dbeta, uint32_t R0, uint32_t cap,
                            uint64_t seed, uint32_t instance, uint32_t step, uint32_t *counts, uint64_t *R_new)
{
    int64_t Emin;
    double lnQ = orc_lnQ(R_prev, E, dbeta, &Emin);
    int s = 63 - orc_ceil_log2(cap);
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * R_prev);
    uint64_t C = 0;
    for (uint32_t j = 0; j < R_prev; ++j) {
        W[j] = (uint64_t)floor(ldexp(exp(-(dbeta * (double)(E[j] - Emin))), s));
        C += W[j];
    }
    uint64_t total = 0;
    for (uint32_t j = 0; j < R_prev; ++j) {
        double tau = (double)((uint64_t)R0 * W[j]) / (double)C;
        counts[j] = orc_poisson_copies(tau, seed, instance, step, j);
        total += counts[j];
    }
    free(W);
    *R_new = total;
    return lnQ;
}

/* Children of parent j occupy consecutive slots, parents in increasing order. */
void orc_children_order(uint32_t R, const uint32_t *counts, uint32_t *parent_of_slot)
{
    uint32_t m = 0;
    for (uint32_t j = 0; j < R; ++j)
        for (uint32_t c = 0; c < counts[j]; ++c) parent_of_slot[m++] = j;
}

/* ------------------------------------------------------------------------ */
/* Population annealing, the Sec. 5.4 algorithm, for one instance.            */
/*   betas[0..S]: beta_0 = 0 (step 1: random start is exact equilibrium),     */
/*   then for i = 1..S: resample to beta_i, theta sweeps at beta_i with sweep  */
/*   counters (i-1) theta ... i theta - 1, measure population averages.       */
/* spins[R*N] in/out: if init != 0 the population is initialised here.       */
/* Per step outputs (arrays of S+1, index 0 = beta_0): lnQ, lnZ, sum E,      */
/* sum E^2 (as double of exact int64 sums), sum |M|, sum M^2, and a running   */
/* FNV-1a hash of the counts; optionally the last step's slot -> parent map   */
/* and every step's energies E_steps[S+1][R]. msc != 0: the sweeps take the  */
/* multi-spin-coded random numbers (reading R18).                             */
/* ------------------------------------------------------------------------ */
void orc_pa_run(int dim, int L, const int8_t *J, uint64_t seed, uint32_t instance, uint32_t R,
                uint32_t S, const double *betas, uint32_t theta, int8_t *spins, int init,
                double *lnQ_out, double *lnZ_out, int64_t *sumE_out, double *sumE2_out,
                int64_t *sumAbsM_out, double *sumM2_out, uint64_t *counts_hash_out,
                int64_t *E_final, int64_t *M_final, uint32_t *parents_last, int64_t *E_steps, int msc)
{
    int64_t N = orc_nsites(dim, L);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * R);
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * R);
    uint32_t *counts = (uint32_t *)malloc(sizeof(uint32_t) * R);
    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * R);
    int8_t *next = (int8_t *)malloc((size_t)R * (size_t)N);

    if (init)
        for (uint32_t r = 0; r < R; ++r)
            orc_init_spins(dim, L, seed, instance, r, 1, spins + (size_t)r * N);

    double lnZ = (double)N * log(2.0);
    uint64_t hash = 1469598103934665603ull;
    for (uint32_t i = 0; i <= S; ++i) {
        double lnQ = 0.0;
        if (i > 0) {
            double dbeta = betas[i] - betas[i - 1];
            lnQ = orc_resample(R, E, dbeta, seed, instance, i, counts);
            for (uint32_t j = 0; j < R; ++j) {
                hash ^= counts[j];
                hash *= 1099511628211ull;
            }
            orc_children_order(R, counts, parent);
            if (parents_last) memcpy(parents_last, parent, sizeof(uint32_t) * R);
            for (uint32_t m = 0; m < R; ++m)
                memcpy(next + (size_t)m * N, spins + (size_t)parent[m] * N, (size_t)N);
            memcpy(spins, next, (size_t)R * (size_t)N);
            for (uint32_t r = 0; r < R; ++r) {
                if (msc)
                    orc_msc_sweeps(dim, L, spins + (size_t)r * N, J, betas[i], seed, instance, r,
                                   (i - 1) * theta, theta);
                else
                    orc_sweeps(dim, L, spins + (size_t)r * N, J, betas[i], seed, instance, r,
                               (i - 1) * theta, theta);
            }
            lnZ += lnQ;
        }
        int64_t sE = 0, sAM = 0;
        double sE2 = 0.0, sM2 = 0.0;
        for (uint32_t r = 0; r < R; ++r) {
            orc_observables(dim, L, spins + (size_t)r * N, J, &E[r], &M[r]);
            sE += E[r];
            sE2 += (double)E[r] * (double)E[r];
            sAM += M[r] < 0 ? -M[r] : M[r];
            sM2 += (double)M[r] * (double)M[r];
        }
        if (E_steps) memcpy(E_steps + (size_t)i * R, E, sizeof(int64_t) * R);
        if (lnQ_out) lnQ_out[i] = lnQ;
        if (lnZ_out) lnZ_out[i] = lnZ;
        if (sumE_out) sumE_out[i] = sE;
        if (sumE2_out) sumE2_out[i] = sE2;
        if (sumAbsM_out) sumAbsM_out[i] = sAM;
        if (sumM2_out) sumM2_out[i] = sM2;
        if (counts_hash_out) counts_hash_out[i] = hash;
    }
    if (E_final) memcpy(E_final, E, sizeof(int64_t) * R);
    if (M_final) memcpy(M_final, M, sizeof(int64_t) * R);
    free(E);
    free(M);
    free(counts);
    free(parent);
    free(next);
}

/* Population annealing (Sec. 5.4) with nearest-integer resampling and a
 * variable population size (reading R17): R_0 = R0 replicas at beta_0, at most
 * cap at any step. spins[cap*N]; the first R_i slots hold the population after
 * step i. Per step: lnQ, lnZ, sum E over the population and its size R_i;
 * E_final[cap] / parents_last[cap] for the last step's first R_S slots.
 * Returns 0, or -1 (outputs up to that step valid) if a step would need more
 * than cap replicas or would leave none. msc != 0: multi-spin-coded sweeps;
 * poisson != 0: Poisson instead of nearest-integer counts (reading R20). */
int orc_pa_run_nearest(int dim, int L, const int8_t *J, uint64_t seed, uint32_t instance, uint32_t R0,
                       uint32_t cap, uint32_t S, const double *betas, uint32_t theta, int8_t *spins, int init,
                       double *lnQ_out, double *lnZ_out, int64_t *sumE_out, uint32_t *nrep_out,
                       int64_t *E_final, uint32_t *parents_last, int msc, int poisson)
{
    int64_t N = orc_nsites(dim, L);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * cap);
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * cap);
    uint32_t *counts = (uint32_t *)malloc(sizeof(uint32_t) * cap);
    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * cap);
    int8_t *next = (int8_t *)malloc((size_t)cap * (size_t)N);
    int rc = 0;

    if (init)
        for (uint32_t r = 0; r < R0; ++r)
            orc_init_spins(dim, L, seed, instance, r, 1, spins + (size_t)r * N);

    uint32_t R = R0;
    double lnZ = (double)N * log(2.0);
    for (uint32_t i = 0; i <= S; ++i) {
        double lnQ = 0.0;
        if (i > 0) {
            double dbeta = betas[i] - betas[i - 1];
            uint64_t Rn;
            lnQ = poisson ? orc_resample_poisson(R, E, dbeta, R0, cap, seed, instance, i, counts, &Rn)
                          : orc_resample_nearest(R, E, dbeta, R0, cap, seed, instance, i, counts, &Rn);
            if (Rn > cap || Rn == 0) {  /* outgrown the capacity, or died out */
                rc = -1;
                break;
            }
            orc_children_order(R, counts, parent);
            R = (uint32_t)Rn;
            if (parents_last) memcpy(parents_last, parent, sizeof(uint32_t) * R);
            for (uint32_t m = 0; m < R; ++m)
                memcpy(next + (size_t)m * N, spins + (size_t)parent[m] * N, (size_t)N);
            memcpy(spins, next, (size_t)R * (size_t)N);
            for (uint32_t r = 0; r < R; ++r) {
                if (msc)
                    orc_msc_sweeps(dim, L, spins + (size_t)r * N, J, betas[i], seed, instance, r,
                                   (i - 1) * theta, theta);
                else
                    orc_sweeps(dim, L, spins + (size_t)r * N, J, betas[i], seed, instance, r,
                               (i - 1) * theta, theta);
            }
            lnZ += lnQ;
        }
        int64_t sE = 0;
        for (uint32_t r = 0; r < R; ++r) {
            orc_observables(dim, L, spins + (size_t)r * N, J, &E[r], &M[r]);
            sE += E[r];
        }
        if (lnQ_out) lnQ_out[i] = lnQ;
        if (lnZ_out) lnZ_out[i] = lnZ;
        if (sumE_out) sumE_out[i] = sE;
        if (nrep_out) nrep_out[i] = R;
    }
    if (E_final) memcpy(E_final, E, sizeof(int64_t) * R);
    free(E);
    free(M);
    free(counts);
    free(parent);
    free(next);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Swendsen-Wang cluster update of the ferromagnet (Sec. 3.3, its three       */
/* steps; reading R19).                                                       */
/*  1. bond b = dim * i + mu (forward bond of site i along axis mu) is active */
/*     iff s_i = s_j and u <= T_bond, u its Philox word (purpose SW_BOND 6,   */
/*     counter (b >> 2, t, replica, c3), word b & 3), T_bond =               */
/*     ceil(p 2^32) - 1 with p = 1 - exp(-2 beta) (so "r < p" as in R2);      */
/*  2. clusters = connected components of the active bonds, each named by its */
/*     smallest site index (found here by breadth-first search from the       */
/*     sites in increasing order);                                            */
/*  3. a cluster flips iff the top bit of the Philox word of its name r       */
/*     (purpose SW_FLIP 7, counter (r >> 2, t, replica, c3), word r & 3) is 1.*/
/* label (may be NULL): [N] the cluster name of every site.                   */
/* ------------------------------------------------------------------------ */
int64_t orc_sw_bond_threshold(double beta)
{
    double p = 1.0 - exp(-2.0 * beta);
    return (int64_t)ceil(ldexp(p, 32)) - 1;
}

/* Step 1: active[dim * i + mu] of every forward bond. */
void orc_sw_bonds(int dim, int L, const int8_t *s, double beta, uint64_t seed, uint32_t instance,
                  uint32_t replica, uint32_t t, uint8_t *active)
{
    int64_t N = orc_nsites(dim, L);
    int64_t Tb = orc_sw_bond_threshold(beta);
    uint32_t cb = orc_c3(ORC_PURPOSE_SW_BOND, 0u, instance);
    for (int64_t i = 0; i < N; ++i)
        for (int mu = 0; mu < dim; ++mu) {
            int Jn;
            int64_t j = orc_neighbour(dim, L, i, 2 * mu, NULL, &Jn);
            int64_t b = (int64_t)dim * i + mu;
            uint32_t u = orc_word(seed, (uint32_t)(b >> 2), t, replica, cb, (unsigned)(b & 3));
            active[b] = (uint8_t)(s[i] == s[j] && (int64_t)u <= Tb);
        }
}

void orc_sw_update(int dim, int L, int8_t *s, double beta, uint64_t seed, uint32_t instance, uint32_t replica,
                   uint32_t t, int32_t *label)
{
    int64_t N = orc_nsites(dim, L);
    uint8_t *active = (uint8_t *)malloc((size_t)N * (dim == 3 ? 3u : 2u));
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    uint32_t cf = orc_c3(ORC_PURPOSE_SW_FLIP, 0u, instance);

    /* 1. bond variables */
    orc_sw_bonds(dim, L, s, beta, seed, instance, replica, t, active);
    /* 2. connected components, named by their smallest site */
    for (int64_t i = 0; i < N; ++i) lab[i] = -1;
    for (int64_t root = 0; root < N; ++root) {
        if (lab[root] >= 0) continue;
        int64_t head = 0, tail = 0;
        lab[root] = (int32_t)root;
        queue[tail++] = root;
        while (head < tail) {
            int64_t i = queue[head++];
            for (int n = 0; n < 2 * dim; ++n) {
                int Jn;
                int64_t j = orc_neighbour(dim, L, i, n, NULL, &Jn);
                int64_t b = (n % 2 == 0) ? (int64_t)dim * i + n / 2 : (int64_t)dim * j + n / 2;
                if (active[b] && lab[j] < 0) {
                    lab[j] = (int32_t)root;
                    queue[tail++] = j;
                }
            }
        }
    }
    /* 3. flip every cluster with probability 1/2 */
    for (int64_t i = 0; i < N; ++i) {
        int64_t r = lab[i];
        uint32_t w = orc_word(seed, (uint32_t)(r >> 2), t, replica, cf, (unsigned)(r & 3));
        if (w >> 31) s[i] = (int8_t)(-s[i]);
        if (label) label[i] = lab[i];
    }
    free(active);
    free(lab);
    free(queue);
}

/* Batch form of the generator for tests: n counters, one key. */
void orc_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Parallel tempering (Sec. 5.1, Eq. (10)) of T replicas of one instance.     */
/* Temperature k has inverse temperature betas[k] (ascending); rep_of[k] is   */
/* the configuration currently at temperature k. One step: theta sweeps of    */
/* every configuration r at the beta of its temperature (sweep counters       */
/* t0 + step*theta + s, replica index r), its energy, then one exchange round */
/* over the pairs (k, k+1) with k = round mod 2, 4, ... Pair (k, k+1) holding  */
/* configurations a, b is swapped with probability min(1, e^D),               */
/* D = (beta_k - beta_{k+1}) (E_a - E_b): always if E_b >= E_a, else iff the   */
/* pair's 32-bit word u (purpose 4: q = k>>2, word k&3, t = round, r = 0)     */
/* satisfies u <= ceil(exp(-(dbeta (E_a - E_b))) 2^32) - 1 (reading R2).      */
/* Swaps exchange temperature labels, not configurations.                     */
/* ------------------------------------------------------------------------ */
void orc_pt_run(int dim, int L, const int8_t *J, uint64_t seed, uint32_t instance, uint32_t T,
                const double *betas, uint32_t theta, uint32_t n_steps, uint32_t t0, uint32_t round0,
                int8_t *spins, uint32_t *rep_of, uint32_t *accepted, int64_t *E_out)
{
    int64_t N = orc_nsites(dim, L);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * T);
    uint32_t *temp_of = (uint32_t *)malloc(sizeof(uint32_t) * T);
    for (uint32_t k = 0; k < T; ++k) temp_of[rep_of[k]] = k;
    for (uint32_t step = 0; step < n_steps; ++step) {
        for (uint32_t r = 0; r < T; ++r) {
            orc_sweeps(dim, L, spins + (size_t)r * N, J, betas[temp_of[r]], seed, instance, r,
                       t0 + step * theta, theta);
            int64_t M;
            orc_observables(dim, L, spins + (size_t)r * N, J, &E[r], &M);
        }
        uint32_t round = round0 + step;
        for (uint32_t k = round % 2; k + 1 < T; k += 2) {
            uint32_t a = rep_of[k], b = rep_of[k + 1];
            int accept;
            if (E[b] >= E[a]) {
                accept = 1;
            } else {
                double dbeta = betas[k + 1] - betas[k];
                double p = exp(-(dbeta * (double)(E[a] - E[b])));
                int64_t thr = (int64_t)ceil(ldexp(p, 32)) - 1;
                uint32_t u = orc_word(seed, k >> 2, round, 0u, (4u << 28) | instance, k & 3u);
                accept = (int64_t)u <= thr;
            }
            if (accept) {
                rep_of[k] = b;
                rep_of[k + 1] = a;
                temp_of[b] = k;
                temp_of[a] = k + 1;
                accepted[k] += 1;
            }
        }
    }
    if (E_out) memcpy(E_out, E, sizeof(int64_t) * T);
    free(E);
    free(temp_of);
}
