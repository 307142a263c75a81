/*
 * pgg_oracle.c -- CPU oracle for the spatial public goods game Monte Carlo of
 * M. Perc, "High-performance parallel computing in the classroom using the public
 * goods game as an example" (arXiv:1704.08098).
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain, obviously-correct statement
 * of what the GPU library computes. Only the tests, the smoke check and the CPU
 * baseline of the benchmark load it; the product path never does. It shares no
 * code, header, table or constant generator with the CUDA library: the random
 * stream layout and the threshold rule below are restated here from their written
 * definitions, independently of the library's own implementation.
 *
 * What it computes
 *   - Section III, Eq. (1)-(2): the payoff of a player from each of the G = 5
 *     overlapping groups it belongs to (Fig. 1), summed over the groups.
 *   - Eq. (3): the Fermi probability W = 1 / (1 + exp((P_x - P_y) / K)) that x
 *     adopts the strategy of its randomly chosen neighbour y, turned into a uint32
 *     threshold t so that "adopt iff u < t" for a uint32 random draw u.
 *   - Section III: initial condition (each site C or D with probability 1/2, or p).
 *   - The elementary step made parallel by a fixed schedule: step k updates every
 *     site whose (row mod 4, column mod 4) equals an offset drawn for that step;
 *     16 steps are one full Monte Carlo step (MCS, Section III: L^2 elementary
 *     updates). Concurrent sites are at Manhattan distance >= 4, so the radius-3
 *     read set of one update (Section IV, Fig. 3: a halo three rows deep) never
 *     contains another update's site; the sites of one step are therefore updated
 *     here one after the other, in row-major order (or reversed, for the
 *     order-independence pin).
 *   - Eq. (4): the cooperator count after every MCS.
 *   - The classic random-sequential dynamics of Section III (a uniformly random
 *     site per elementary step), used only as a statistical reference.
 *   - Section VI: the same scheme for a game played pairwise, not in groups (the
 *     prisoner's dilemma is the example named there): every player plays a 2x2
 *     matrix game with each of its four nearest neighbours. The read set of an
 *     update then shrinks by one line in every direction (radius 2); the schedule,
 *     the random stream and the Fermi rule stay the same.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed low 32 bits, seed high 32
 * bits). Counter layout (c0, c1, c2, c3), tag in bits 24..31 of c3:
 *   init    tag 1: (q_lo, q_hi, 0, 1<<24), q = site >> 2, site = i*L + j;
 *                  word (site & 3); s = C iff word < floor(p * 2^32).
 *   offset  tag 2: (m_lo, m_hi, 0, 2<<24), m = k >> 5; word (k >> 3) & 3;
 *                  o = (word >> 4*(k & 7)) & 15; row offset o >> 2, column o & 3.
 *   dir     tag 3: (b >> 6, a, k_lo, k_hi | 3<<24); word (b >> 4) & 3;
 *                  d = (word >> 2*(b & 15)) & 3; 0: j+1, 1: j-1, 2: i+1, 3: i-1.
 *   u       tag 4: (b >> 2, a, k_lo, k_hi | 4<<24); u = word (b & 3).
 *   classic tag 5: (e_lo, e_hi, 0, 5<<24) for elementary step e.
 * where k is the sublattice step index (k < 2^56), and (a, b) are the sublattice
 * coordinates of site (i, j) = (4a + row offset, 4b + column offset).
 *
 * Threshold (the reading used for bit-exact parity): with S the sum of the
 * cooperator counts of the five groups of a player, the sum of Eq. (1)-(2) over
 * its groups is P(s, S) = (r*S)/5 - 5*s (c = 1, G = 5). The oracle evaluates the
 * payoff group by group as printed and checks that it equals P(s, S); the
 * threshold is formed from P(s, S) in IEEE double precision with no contraction:
 *   D = P(s_x, S_x) - P(s_y, S_y);  W = 1/(1 + exp(D/K));
 *   t = (W >= 1) ? 2^32 - 1 : floor(W * 2^32);  adopt iff s_x != s_y and u < t.
 *
 * Pairwise game (reading of Section VI, which names the game but prints no
 * payoffs): pay = {R, S, T, P} is the payoff of a cooperator meeting a cooperator
 * (R) or a defector (S), and of a defector meeting a cooperator (T) or a defector
 * (P). With n the number of cooperators among the four neighbours, the sum over
 * the four games is P(s, n) = n*A + (4 - n)*B, (A, B) = (R, S) for s = C and
 * (T, P) for s = D; the oracle sums game by game, checks it against P(s, n) and
 * forms the threshold from P(s, n) exactly as above.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp].
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11).                                     */
/* One round: two 32x32->64 products of the multipliers with counter words 0  */
/* and 2; the high halves are xored with the other two counter words and the  */
/* key; words are permuted; the key advances by the Weyl constants.           */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

enum { TAG_INIT = 1, TAG_OFFSET = 2, TAG_DIR = 3, TAG_U = 4, TAG_CLASSIC = 5 };

/* Offset of sublattice step k: 0..15, row offset = o >> 2, column offset = o & 3. */
int oracle_offset(uint64_t seed, uint64_t k)
{
    uint64_t m = k >> 5;
    uint32_t w[4];
    philox_seeded(seed, (uint32_t)m, (uint32_t)(m >> 32), 0u, (uint32_t)TAG_OFFSET << 24, w);
    uint32_t word = w[(k >> 3) & 3];
    return (int)((word >> (4 * (k & 7))) & 15u);
}

/* Neighbour direction for sublattice site (a, b) at step k. */
int oracle_dir(uint64_t seed, uint64_t k, uint32_t a, uint32_t b)
{
    uint32_t w[4];
    philox_seeded(seed, b >> 6, a, (uint32_t)k, (uint32_t)(k >> 32) | ((uint32_t)TAG_DIR << 24), w);
    uint32_t word = w[(b >> 4) & 3];
    return (int)((word >> (2 * (b & 15))) & 3u);
}

/* Adoption draw for sublattice site (a, b) at step k. */
uint32_t oracle_u(uint64_t seed, uint64_t k, uint32_t a, uint32_t b)
{
    uint32_t w[4];
    philox_seeded(seed, b >> 2, a, (uint32_t)k, (uint32_t)(k >> 32) | ((uint32_t)TAG_U << 24), w);
    return w[b & 3];
}

/* ------------------------------------------------------------------------- */
/* The game (Section III, Fig. 1, Eq. (1)-(2)).                               */
/* ------------------------------------------------------------------------- */
static int wrap(int v, int L) { return ((v % L) + L) % L; }

static int strategy_at(const uint8_t *lat, int L, int i, int j)
{
    return lat[(size_t)wrap(i, L) * (size_t)L + (size_t)wrap(j, L)] ? 1 : 0;
}

/* The four von Neumann neighbours, in the order of the direction code. */
static const int NB_DI[4] = {0, 0, 1, -1};
static const int NB_DJ[4] = {1, -1, 0, 0};

/* Number of cooperators N_C in the group of G = 5 centred on (ci, cj): the centre
 * and its four nearest neighbours (Fig. 1). Sites repeated by the periodic wrap on
 * tiny lattices are counted once per appearance. */
int oracle_group_cooperators(const uint8_t *lat, int L, int ci, int cj)
{
    int n = strategy_at(lat, L, ci, cj);
    for (int d = 0; d < 4; ++d)
        n += strategy_at(lat, L, ci + NB_DI[d], cj + NB_DJ[d]);
    return n;
}

/* Payoff of the player at (i, j) summed over its five groups, group by group as
 * Eq. (1) (cooperator: r*c*N_C/G - c) and Eq. (2) (defector: r*c*N_C/G), c = 1,
 * G = 5. The groups are the one centred on the player and the four centred on its
 * neighbours (Fig. 1). */
double oracle_payoff_groups(const uint8_t *lat, int L, int i, int j, double r)
{
    const double G = 5.0, c = 1.0;
    int s = strategy_at(lat, L, i, j);
    double pi = 0.0;
    for (int g = 0; g < 5; ++g) {
        int ci = (g == 0) ? i : i + NB_DI[g - 1];
        int cj = (g == 0) ? j : j + NB_DJ[g - 1];
        int nc = oracle_group_cooperators(lat, L, ci, cj);
        double share = r * c * (double)nc / G;
        pi += s ? (share - c) : share;
    }
    return pi;
}

/* Sum over the player's five groups of their cooperator counts, S in [0, 25]. */
int oracle_group_count_total(const uint8_t *lat, int L, int i, int j)
{
    int S = oracle_group_cooperators(lat, L, i, j);
    for (int d = 0; d < 4; ++d)
        S += oracle_group_cooperators(lat, L, i + NB_DI[d], j + NB_DJ[d]);
    return S;
}

/* The same payoff from the integer total: sum_g (r N_g / 5 - s) = r S / 5 - 5 s. */
double oracle_payoff_total(int s, int S, double r)
{
    return (r * (double)S) / 5.0 - 5.0 * (double)s;
}

/* Eq. (3) as a uint32 threshold: x adopts s_y iff a uniform uint32 u < t. */
uint32_t oracle_fermi_threshold(double pi_x, double pi_y, double K)
{
    double W = 1.0 / (1.0 + exp((pi_x - pi_y) / K));
    if (W >= 1.0)
        return 0xFFFFFFFFu;
    return (uint32_t)(W * 4294967296.0);
}

static int g_error = 0;

/* Count of internal consistency failures (group-by-group payoff vs the total). */
int oracle_error_count(void) { return g_error; }
void oracle_clear_errors(void) { g_error = 0; }

/* The adoption of Eq. (3): x takes the strategy s_y of y iff u < t. */
static int adopt(uint8_t *lat, int L, int i, int j, int sy, uint32_t t, uint32_t u)
{
    if (u < t) {
        lat[(size_t)i * (size_t)L + (size_t)j] = (uint8_t)sy;
        return 1;
    }
    return 0;
}

/* Elementary update of Section III for player x = (i, j) and its neighbour in
 * direction dir, with adoption draw u. Returns 1 if x changed strategy. */
int oracle_elementary_update(uint8_t *lat, int L, int i, int j, int dir, uint32_t u,
                             double r, double K)
{
    int yi = i + NB_DI[dir], yj = j + NB_DJ[dir];
    int sx = strategy_at(lat, L, i, j);
    int sy = strategy_at(lat, L, yi, yj);
    if (sx == sy)
        return 0;
    int Sx = oracle_group_count_total(lat, L, i, j);
    int Sy = oracle_group_count_total(lat, L, yi, yj);
    double px = oracle_payoff_total(sx, Sx, r);
    double py = oracle_payoff_total(sy, Sy, r);
    double gx = oracle_payoff_groups(lat, L, i, j, r);
    double gy = oracle_payoff_groups(lat, L, yi, yj, r);
    if (fabs(gx - px) > 1e-9 * (1.0 + fabs(px)) || fabs(gy - py) > 1e-9 * (1.0 + fabs(py))) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        g_error++;
    }
    uint32_t t = oracle_fermi_threshold(px, py, K);
    return adopt(lat, L, i, j, sy, t, u);
}

/* ------------------------------------------------------------------------- */
/* The pairwise game (Section VI).                                            */
/* ------------------------------------------------------------------------- */

/* Payoff of one game between a player with strategy s and one with s_other. */
static double pair_matrix(int s, int s_other, const double pay[4])
{
    if (s)
        return s_other ? pay[0] : pay[1];
    return s_other ? pay[2] : pay[3];
}

/* Number of cooperators among the four nearest neighbours of (i, j). */
int oracle_pair_neighbour_cooperators(const uint8_t *lat, int L, int i, int j)
{
    int n = 0;
    for (int d = 0; d < 4; ++d)
        n += strategy_at(lat, L, i + NB_DI[d], j + NB_DJ[d]);
    return n;
}

/* Payoff of the player at (i, j), game by game over its four neighbours. */
double oracle_pair_payoff_games(const uint8_t *lat, int L, int i, int j, const double pay[4])
{
    int s = strategy_at(lat, L, i, j);
    double pi = 0.0;
    for (int d = 0; d < 4; ++d)
        pi += pair_matrix(s, strategy_at(lat, L, i + NB_DI[d], j + NB_DJ[d]), pay);
    return pi;
}

/* The same payoff from the count n of cooperating neighbours. */
double oracle_pair_payoff_total(int s, int n, const double pay[4])
{
    double a = s ? pay[0] : pay[2];
    double b = s ? pay[1] : pay[3];
    return (double)n * a + (double)(4 - n) * b;
}

/* Threshold of the update of x = (i, j) towards its neighbour in direction dir
 * (0 when the two already agree). */
uint32_t oracle_pair_update_threshold(const uint8_t *lat, int L, int i, int j, int dir,
                                      const double pay[4], double K)
{
    int yi = i + NB_DI[dir], yj = j + NB_DJ[dir];
    int sx = strategy_at(lat, L, i, j);
    int sy = strategy_at(lat, L, yi, yj);
    if (sx == sy)
        return 0;
    int nx = oracle_pair_neighbour_cooperators(lat, L, i, j);
    int ny = oracle_pair_neighbour_cooperators(lat, L, yi, yj);
    double px = oracle_pair_payoff_total(sx, nx, pay);
    double py = oracle_pair_payoff_total(sy, ny, pay);
    double gx = oracle_pair_payoff_games(lat, L, i, j, pay);
    double gy = oracle_pair_payoff_games(lat, L, yi, yj, pay);
    if (fabs(gx - px) > 1e-9 * (1.0 + fabs(px)) || fabs(gy - py) > 1e-9 * (1.0 + fabs(py))) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        g_error++;
    }
    return oracle_fermi_threshold(px, py, K);
}

/* Elementary update of the pairwise game. Returns 1 if x changed strategy. */
int oracle_pair_elementary_update(uint8_t *lat, int L, int i, int j, int dir, uint32_t u,
                                  const double pay[4], double K)
{
    int sy = strategy_at(lat, L, i + NB_DI[dir], j + NB_DJ[dir]);
    if (strategy_at(lat, L, i, j) == sy)
        return 0;
    uint32_t t = oracle_pair_update_threshold(lat, L, i, j, dir, pay, K);
    return adopt(lat, L, i, j, sy, t, u);
}

/* Which game an update plays: the group game with synergy r, or the pairwise
 * game with matrix pay. */
struct game {
    int pairwise;
    double r;
    double pay[4];
};

static int game_update(uint8_t *lat, int L, int i, int j, int dir, uint32_t u,
                       const struct game *g, double K)
{
    if (g->pairwise)
        return oracle_pair_elementary_update(lat, L, i, j, dir, u, g->pay, K);
    return oracle_elementary_update(lat, L, i, j, dir, u, g->r, K);
}

/* ------------------------------------------------------------------------- */
/* Dynamics.                                                                  */
/* ------------------------------------------------------------------------- */

/* Initial condition (Section III): site C with probability p, independently. */
void oracle_init(uint8_t *lat, int L, uint64_t seed, double p)
{
    uint64_t thr = (uint64_t)(p * 4294967296.0);
    if (p >= 1.0) thr = 4294967296ull;
    if (p <= 0.0) thr = 0;
    uint64_t n = (uint64_t)L * (uint64_t)L;
    for (uint64_t x = 0; x < n; ++x) {
        uint64_t q = x >> 2;
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)q, (uint32_t)(q >> 32), 0u, (uint32_t)TAG_INIT << 24, w);
        lat[x] = ((uint64_t)w[x & 3] < thr) ? 1 : 0;
    }
}

/* Number of cooperators on the lattice (numerator of Eq. (4)). */
uint64_t oracle_count(const uint8_t *lat, int L)
{
    uint64_t n = (uint64_t)L * (uint64_t)L, c = 0;
    for (uint64_t x = 0; x < n; ++x)
        c += lat[x] ? 1 : 0;
    return c;
}

/* One sublattice step k: every site with (i mod 4, j mod 4) equal to the drawn
 * offset makes one elementary update. reverse != 0 visits the sites in reverse
 * order; threads > 1 splits the sublattice rows over OpenMP threads (the sites
 * are independent, so all three give the same lattice). Returns the number of
 * adoptions. */
static int64_t game_sublattice_step(uint8_t *lat, int L, const struct game *g, double K,
                                    uint64_t seed, uint64_t k, int reverse, int threads)
{
    int o = oracle_offset(seed, k);
    int oi = o >> 2, oj = o & 3;
    int n4 = L / 4;
    int64_t changed = 0;
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads > 0 ? threads : 1) reduction(+ : changed) schedule(static) if (threads > 1)
#endif
    for (int aa = 0; aa < n4; ++aa) {
        int a = reverse ? (n4 - 1 - aa) : aa;
        for (int bb = 0; bb < n4; ++bb) {
            int b = reverse ? (n4 - 1 - bb) : bb;
            int i = 4 * a + oi, j = 4 * b + oj;
            int d = oracle_dir(seed, k, (uint32_t)a, (uint32_t)b);
            uint32_t u = oracle_u(seed, k, (uint32_t)a, (uint32_t)b);
            changed += game_update(lat, L, i, j, d, u, g, K);
        }
    }
    return changed;
}

/* n_mcs full Monte Carlo steps (16 sublattice steps each) starting at sublattice
 * step k0; counts[m] (if not NULL) receives the cooperator count after MCS m.
 * Returns 0, or -1 for an invalid lattice size. */
static int game_run(uint8_t *lat, int L, const struct game *g, double K, uint64_t seed,
                    uint64_t k0, int64_t n_mcs, uint64_t *counts, int reverse, int threads)
{
    if (L < 4 || L % 4 != 0)
        return -1;
    uint64_t k = k0;
    for (int64_t m = 0; m < n_mcs; ++m) {
        for (int s = 0; s < 16; ++s, ++k)
            game_sublattice_step(lat, L, g, K, seed, k, reverse, threads);
        if (counts)
            counts[m] = oracle_count(lat, L);
    }
    return 0;
}

/* Classic random-sequential dynamics exactly as described in Section III: each
 * elementary step picks a uniformly random site and a uniformly random neighbour;
 * L^2 elementary steps form one MCS. Statistical reference only (its stream, tag
 * 5, is not shared with the parallel schedule). e0 is the first elementary-step
 * index. */
static int game_classic_run(uint8_t *lat, int L, const struct game *g, double K, uint64_t seed,
                            uint64_t e0, int64_t n_mcs, uint64_t *counts)
{
    if (L < 3)
        return -1;
    uint64_t n = (uint64_t)L * (uint64_t)L;
    uint64_t e = e0;
    for (int64_t m = 0; m < n_mcs; ++m) {
        for (uint64_t t = 0; t < n; ++t, ++e) {
            uint32_t w[4];
            philox_seeded(seed, (uint32_t)e, (uint32_t)(e >> 32), 0u, (uint32_t)TAG_CLASSIC << 24, w);
            uint64_t r64 = ((uint64_t)w[0] << 32) | w[1];
            uint64_t x = (uint64_t)(((unsigned __int128)r64 * n) >> 64);
            int i = (int)(x / (uint64_t)L), j = (int)(x % (uint64_t)L);
            int d = (int)(w[2] >> 30);
            game_update(lat, L, i, j, d, w[3], g, K);
        }
        if (counts)
            counts[m] = oracle_count(lat, L);
    }
    return 0;
}

static struct game group_game(double r)
{
    struct game g = {0, r, {0.0, 0.0, 0.0, 0.0}};
    return g;
}

static struct game pair_game(const double pay[4])
{
    struct game g = {1, 0.0, {pay[0], pay[1], pay[2], pay[3]}};
    return g;
}

/* The public goods game (Section III) ... */
int64_t oracle_sublattice_step(uint8_t *lat, int L, double r, double K, uint64_t seed,
                               uint64_t k, int reverse, int threads)
{
    struct game g = group_game(r);
    return game_sublattice_step(lat, L, &g, K, seed, k, reverse, threads);
}

int oracle_run(uint8_t *lat, int L, double r, double K, uint64_t seed, uint64_t k0,
               int64_t n_mcs, uint64_t *counts, int reverse, int threads)
{
    struct game g = group_game(r);
    return game_run(lat, L, &g, K, seed, k0, n_mcs, counts, reverse, threads);
}

int oracle_classic_run(uint8_t *lat, int L, double r, double K, uint64_t seed, uint64_t e0,
                       int64_t n_mcs, uint64_t *counts)
{
    struct game g = group_game(r);
    return game_classic_run(lat, L, &g, K, seed, e0, n_mcs, counts);
}

/* ... and the pairwise game (Section VI), on the same schedule and stream. */
int64_t oracle_pair_sublattice_step(uint8_t *lat, int L, const double pay[4], double K,
                                    uint64_t seed, uint64_t k, int reverse, int threads)
{
    struct game g = pair_game(pay);
    return game_sublattice_step(lat, L, &g, K, seed, k, reverse, threads);
}

int oracle_pair_run(uint8_t *lat, int L, const double pay[4], double K, uint64_t seed,
                    uint64_t k0, int64_t n_mcs, uint64_t *counts, int reverse, int threads)
{
    struct game g = pair_game(pay);
    return game_run(lat, L, &g, K, seed, k0, n_mcs, counts, reverse, threads);
}

int oracle_pair_classic_run(uint8_t *lat, int L, const double pay[4], double K, uint64_t seed,
                            uint64_t e0, int64_t n_mcs, uint64_t *counts)
{
    struct game g = pair_game(pay);
    return game_classic_run(lat, L, &g, K, seed, e0, n_mcs, counts);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
