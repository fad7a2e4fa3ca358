/*
 * Oracle noise sampler: i.i.d. single-qubit Pauli channel drawn from the
 * counter-based Philox4x64-10 generator, and the syndrome s = <H, E>.
 *
 * TEST INFRASTRUCTURE ONLY (see bp_oracle.c).  It shares no code with the
 * CUDA path; both sides implement the same published generator.
 *
 *  - Channel: each qubit independently suffers X, Y, Z with probabilities
 *    p^X, p^Y, p^Z and no error otherwise.  The depolarising channel of
 *    Sec. IV (each of X, Y, Z with probability p/3) and the Z-biased channel
 *    of Sec. IV-B3 are special cases.
 *  - Generator: Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw,
 *    "Parallel random numbers: as easy as 1, 2, 3", SC 2011).  Key =
 *    (seed, 0).  Counter = (shot, j / 4, 0, 0); output word j % 4 is the
 *    draw u of qubit j.
 *  - A draw becomes a Pauli by comparing u with the integer thresholds
 *    T_X = floor(p^X 2^64), T_Y = floor((p^X + p^Y) 2^64),
 *    T_Z = floor((p^X + p^Y + p^Z) 2^64), the sums taken in double in that
 *    order: u < T_X -> X, else u < T_Y -> Y, else u < T_Z -> Z, else I.
 *  - Syndrome: s_i = XOR_j <E_j, H_ij>, the trace inner product (1 when the
 *    two Paulis anticommute), Sec. II-A.
 *
 * Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z.
 */
#include <math.h>
#include <stdint.h>

#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One Philox4x64-10 block: out = philox(ctr, key). */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(PHILOX_M0, x0, &hi0, &lo0);
        mulhilo64(PHILOX_M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* floor(c * 2^64) for 0 <= c < 1. */
static uint64_t threshold(double c) {
    if (c <= 0.0) return 0;
    return (uint64_t)ldexp(c, 64);
}

static int anticommutes(int a, int b) { return a != 0 && b != 0 && a != b; }

/* Draw B shots (shot indices shot0 .. shot0+B-1) of the i.i.d. Pauli channel
 * on N qubits and their syndromes for the M x N Pauli check matrix H.
 * err: B x N codes; syn: B x M bytes (0/1). */
int oracle_sample(int N, int M, const uint8_t *H, double px, double py, double pz, uint64_t seed,
                  uint64_t shot0, int B, uint8_t *err, uint8_t *syn) {
    if (N <= 0 || M < 0 || B < 0) return -1;
    if (!(px >= 0 && py >= 0 && pz >= 0)) return -1;
    double cx = px, cy = cx + py, cz = cy + pz;
    if (!(cz < 1.0)) return -1;
    uint64_t tx = threshold(cx), ty = threshold(cy), tz = threshold(cz);
    uint64_t key[2] = {seed, 0};
    for (int b = 0; b < B; ++b) {
        uint8_t *e = err + (long)b * N;
        for (int j = 0; j < N; ++j) {
            uint64_t ctr[4] = {shot0 + (uint64_t)b, (uint64_t)(j / 4), 0, 0}, out[4];
            oracle_philox4x64_10(ctr, key, out);
            uint64_t u = out[j % 4];
            e[j] = u < tx ? 1 : u < ty ? 2 : u < tz ? 3 : 0;
        }
        uint8_t *s = syn + (long)b * M;
        for (int i = 0; i < M; ++i) {
            int par = 0;
            for (int j = 0; j < N; ++j) par ^= anticommutes(e[j], H[(long)i * N + j]);
            s[i] = (uint8_t)par;
        }
    }
    return 0;
}
