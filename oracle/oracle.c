/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the state-vector
 * hot path of "Deep Quantum Circuit Simulations of Low-energy Nuclear States"
 * (arXiv 2310.17739).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the GPU library: it has its own gate
 * table, its own index arithmetic, its own Philox and its own measurement
 * logic, and nothing from the GPU library ever feeds it.
 *
 * Precision: complex128 (C99 double _Complex) throughout, single-threaded,
 * every sum taken in plain index order.  Built with -ffp-contract=off so that
 * x86-64 and aarch64 hosts give bit-identical results.
 *
 * What each function follows:
 *   og_matrix        gate definitions of the OpenQASM gate table (Table
 *                    "Gates defined in IBM OpenQASM"), with the global-phase
 *                    conventions RZ(t)=exp(-i t Z/2), U1(l)=diag(1,e^{il}),
 *                    U3 as the standard three-angle matrix.
 *   og_apply_1q      Eq. (1q-op): s_i = floor(i/2^q) 2^{q+1} + (i mod 2^q),
 *                    (a_{s_i}, a_{s_i+2^q}) <- U_{2x2} (a_{s_i}, a_{s_i+2^q}).
 *   og_apply_2q      Eq. (2q-op) with p<q the sorted operand pair:
 *                    s_i = floor(floor(i/2^p)/2^{q-p-1}) 2^{q+1}
 *                          + (floor(i/2^p) mod 2^{q-p-1}) 2^{p+1} + (i mod 2^p);
 *                    the four amplitudes of the group are then addressed in
 *                    the gate's own operand order (local index b_q0 + 2 b_q1).
 *   oracle_prob /    Section "Mid-Circuit Measurement Assertion": Born
 *   oracle_measure   probability of the measured qubit, a draw (or the
 *                    assertion that the outcome is 0 while P(0) > thr), collapse
 *                    onto the outcome and renormalisation by 1/sqrt(p_out).
 *   oracle_reset     Listing "Block structure ...": `reset q` after a
 *                    measurement: draw an outcome, collapse, and if it was 1
 *                    move the amplitudes back onto the |0> half.
 *   oracle_expect    <psi| sum_t c_t P_t |psi> written as the plain double sum
 *                    over the nonzero matrix entries of each Pauli string.
 *   oracle_philox    Philox4x64-10, Salmon, Moraes, Dror & Shaw, "Parallel
 *                    random numbers: as easy as 1, 2, 3" (SC'11).  The draw
 *                    u(seed,k) = (word 0 of the block with counter (k,0,0,0)
 *                    and key (seed,0)) >> 11, times 2^-53.
 *   oracle_sample    final-state sampling (the register read-out `measure q
 *                    -> c` of Listing "Block structure ...", taken m times
 *                    from one state without collapse): shot s draws
 *                    v(seed,s) from the block with counter (s,1,0,0) and
 *                    returns the smallest index x with v * total <
 *                    sum_{i<=x} |a_i|^2 (Born rule, cumulative sum in index
 *                    order), the bits of a mask packed in ascending order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cd;

/* Input record layout (an interface the library shares by format only). */
typedef struct {
    uint16_t op;
    uint16_t flags;
    uint32_t q0;
    uint32_t q1;
    uint32_t mat;   /* offset, in doubles, of a C1/C2 matrix inside mats[] */
    double p[3];
} og_gate;

typedef struct {
    uint64_t x;     /* qubits carrying X or Y */
    uint64_t z;     /* qubits carrying Z or Y */
    double coef;
} og_term;

enum {
    OG_ID = 0, OG_X = 1, OG_Y = 2, OG_Z = 3, OG_H = 4, OG_S = 5, OG_SDG = 6,
    OG_T = 7, OG_TDG = 8, OG_RX = 9, OG_RY = 10, OG_RZ = 11, OG_U1 = 12,
    OG_U2 = 13, OG_U3 = 14, OG_C1 = 15,
    OG_CX = 32, OG_CY = 33, OG_CZ = 34, OG_CH = 35, OG_SWAP = 36, OG_CRX = 37,
    OG_CRY = 38, OG_CRZ = 39, OG_CU1 = 40, OG_CU3 = 41, OG_RXX = 42,
    OG_RZZ = 43, OG_C2 = 44,
    OG_MEASURE = 64, OG_RESET = 65, OG_BARRIER = 66
};

enum { OG_OK = 0, OG_E_INVAL = 1, OG_E_ZEROPROB = 4 };

#define OG_MEAS_ASSERT 1u

/* ---------------------------------------------------------------- gates -- */

static void m2(cd *m, cd a, cd b, cd c, cd d) { m[0] = a; m[1] = b; m[2] = c; m[3] = d; }

/* 1-qubit definitions, row-major U[r][c], basis |0>,|1>. */
static int og_matrix_1q(int op, const double *p, cd *u)
{
    const double h = 1.0 / sqrt(2.0);
    switch (op) {
    case OG_ID:  m2(u, 1, 0, 0, 1); return 0;
    case OG_X:   m2(u, 0, 1, 1, 0); return 0;
    case OG_Y:   m2(u, 0, -I, I, 0); return 0;
    case OG_Z:   m2(u, 1, 0, 0, -1); return 0;
    case OG_H:   m2(u, h, h, h, -h); return 0;
    case OG_S:   m2(u, 1, 0, 0, I); return 0;
    case OG_SDG: m2(u, 1, 0, 0, -I); return 0;
    case OG_T:   m2(u, 1, 0, 0, cexp(I * M_PI / 4)); return 0;
    case OG_TDG: m2(u, 1, 0, 0, cexp(-I * M_PI / 4)); return 0;
    case OG_RX: {  /* exp(-i t X / 2) */
        double c = cos(p[0] / 2), s = sin(p[0] / 2);
        m2(u, c, -I * s, -I * s, c); return 0;
    }
    case OG_RY: {  /* exp(-i t Y / 2) */
        double c = cos(p[0] / 2), s = sin(p[0] / 2);
        m2(u, c, -s, s, c); return 0;
    }
    case OG_RZ:    /* exp(-i t Z / 2) */
        m2(u, cexp(-I * p[0] / 2), 0, 0, cexp(I * p[0] / 2)); return 0;
    case OG_U1:
        m2(u, 1, 0, 0, cexp(I * p[0])); return 0;
    case OG_U2: case OG_U3: {
        double th = (op == OG_U2) ? M_PI / 2 : p[0];
        double ph = (op == OG_U2) ? p[0] : p[1];
        double la = (op == OG_U2) ? p[1] : p[2];
        double c = cos(th / 2), s = sin(th / 2);
        m2(u, c, -cexp(I * la) * s, cexp(I * ph) * s, cexp(I * (ph + la)) * c);
        return 0;
    }
    default: return -1;
    }
}

/*
 * 2-qubit definitions in the local basis l = b_q0 + 2*b_q1 (q0 = first operand,
 * the control of controlled gates).  M[r*4 + c].
 */
static int og_matrix_2q(int op, const double *p, cd *m)
{
    memset(m, 0, 16 * sizeof(cd));
    cd u[4];
    int ctrl_op = -1;
    switch (op) {
    case OG_CX:  ctrl_op = OG_X; break;
    case OG_CY:  ctrl_op = OG_Y; break;
    case OG_CZ:  ctrl_op = OG_Z; break;
    case OG_CH:  ctrl_op = OG_H; break;
    case OG_CRX: ctrl_op = OG_RX; break;
    case OG_CRY: ctrl_op = OG_RY; break;
    case OG_CRZ: ctrl_op = OG_RZ; break;
    case OG_CU1: ctrl_op = OG_U1; break;
    case OG_CU3: ctrl_op = OG_U3; break;
    default: break;
    }
    if (ctrl_op >= 0) {
        /* |0><0|_c (x) I  +  |1><1|_c (x) U, control = bit 0 of l, target = bit 1 */
        og_matrix_1q(ctrl_op, p, u);
        for (int bt = 0; bt < 2; bt++)          /* control 0: identity on target */
            m[(0 + 2 * bt) * 4 + (0 + 2 * bt)] = 1;
        for (int to = 0; to < 2; to++)
            for (int ti = 0; ti < 2; ti++)
                m[(1 + 2 * to) * 4 + (1 + 2 * ti)] = u[to * 2 + ti];
        return 0;
    }
    switch (op) {
    case OG_SWAP:
        m[0 * 4 + 0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[3 * 4 + 3] = 1;
        return 0;
    case OG_RXX: {  /* exp(-i t X(x)X / 2) = cos(t/2) I - i sin(t/2) X(x)X */
        double c = cos(p[0] / 2), s = sin(p[0] / 2);
        for (int l = 0; l < 4; l++) {
            m[l * 4 + l] = c;
            m[l * 4 + (l ^ 3)] = -I * s;
        }
        return 0;
    }
    case OG_RZZ: {  /* exp(-i t Z(x)Z / 2): phase by parity of (b0, b1) */
        for (int l = 0; l < 4; l++) {
            int parity = (l & 1) ^ ((l >> 1) & 1);
            m[l * 4 + l] = cexp((parity ? I : -I) * p[0] / 2);
        }
        return 0;
    }
    default: return -1;
    }
}

static int og_is_1q(int op) { return op >= OG_ID && op <= OG_C1; }
static int og_is_2q(int op) { return op >= OG_CX && op <= OG_C2; }

/* Public: matrix of one gate record (2x2 or 4x4, interleaved re/im, row-major).
 * Returns the matrix dimension (2 or 4), or -1 for an unknown/non-unitary op. */
int oracle_gate_matrix(const og_gate *g, const double *mats, double *out)
{
    cd m[16];
    int dim;
    if (og_is_1q(g->op)) {
        dim = 2;
        if (g->op == OG_C1) {
            for (int i = 0; i < 4; i++) m[i] = mats[g->mat + 2 * i] + I * mats[g->mat + 2 * i + 1];
        } else if (og_matrix_1q(g->op, g->p, m) != 0) {
            return -1;
        }
    } else if (og_is_2q(g->op)) {
        dim = 4;
        if (g->op == OG_C2) {
            for (int i = 0; i < 16; i++) m[i] = mats[g->mat + 2 * i] + I * mats[g->mat + 2 * i + 1];
        } else if (og_matrix_2q(g->op, g->p, m) != 0) {
            return -1;
        }
    } else {
        return -1;
    }
    for (int i = 0; i < dim * dim; i++) {
        out[2 * i] = creal(m[i]);
        out[2 * i + 1] = cimag(m[i]);
    }
    return dim;
}

/* --------------------------------------------------- Eq. (1q-op), (2q-op) -- */

static void og_apply_1q(cd *a, int n, int q, const cd *u)
{
    const uint64_t half = (uint64_t)1 << (n - 1);
    const uint64_t bq = (uint64_t)1 << q;
    for (uint64_t i = 0; i < half; i++) {
        uint64_t s = (i / bq) * (2 * bq) + (i % bq);
        cd x0 = a[s], x1 = a[s + bq];
        a[s] = u[0] * x0 + u[1] * x1;
        a[s + bq] = u[2] * x0 + u[3] * x1;
    }
}

static void og_apply_2q(cd *a, int n, int q0, int q1, const cd *m)
{
    const int p = q0 < q1 ? q0 : q1;
    const int q = q0 < q1 ? q1 : q0;
    const uint64_t quarter = (uint64_t)1 << (n - 2);
    const uint64_t bp = (uint64_t)1 << p;
    const uint64_t span = (uint64_t)1 << (q - p - 1);
    const uint64_t off0 = (uint64_t)1 << q0, off1 = (uint64_t)1 << q1;
    for (uint64_t i = 0; i < quarter; i++) {
        uint64_t t = i / bp;
        uint64_t s = (t / span) * ((uint64_t)2 << q) + (t % span) * ((uint64_t)2 << p) + (i % bp);
        uint64_t idx[4] = { s, s + off0, s + off1, s + off0 + off1 };  /* l = b_q0 + 2 b_q1 */
        cd x[4], y[4];
        for (int l = 0; l < 4; l++) x[l] = a[idx[l]];
        for (int r = 0; r < 4; r++) {
            y[r] = 0;
            for (int c = 0; c < 4; c++) y[r] += m[r * 4 + c] * x[c];
        }
        for (int l = 0; l < 4; l++) a[idx[l]] = y[l];
    }
}

/* ------------------------------------------------------------- Philox -- */

static void og_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 r = (unsigned __int128)a * b;
    *hi = (uint64_t)(r >> 64);
    *lo = (uint64_t)r;
}

/* Philox4x64 with 10 rounds (SC'11): multipliers and Weyl key increments as
 * published for the 4x64 variant. */
void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        og_mulhilo64(M0, c0, &hi0, &lo0);
        og_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double oracle_draw(uint64_t seed, uint64_t k)
{
    uint64_t ctr[4] = { k, 0, 0, 0 }, key[2] = { seed, 0 }, out[4];
    oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

double oracle_shot_draw(uint64_t seed, uint64_t s)
{
    uint64_t ctr[4] = { s, 1, 0, 0 }, key[2] = { seed, 0 }, out[4];
    oracle_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

/* ----------------------------------------------------------- sampling -- */

static uint64_t og_pack_bits(uint64_t x, uint64_t mask)
{
    uint64_t r = 0;
    int j = 0;
    for (int b = 0; b < 64; b++)
        if ((mask >> b) & 1) {
            r |= ((x >> b) & 1) << j;
            j++;
        }
    return r;
}

/* Returns 0, or 1 when the cumulative array cannot be allocated. */
int oracle_sample(const double *psi, int n, uint64_t mask, uint64_t shots, uint64_t seed, uint64_t *out)
{
    const cd *a = (const cd *)psi;
    const uint64_t N = (uint64_t)1 << n;
    double *cum = (double *)malloc(N * sizeof(double));
    if (!cum) return 1;
    double acc = 0;
    for (uint64_t i = 0; i < N; i++) {
        acc += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
        cum[i] = acc;
    }
    for (uint64_t s = 0; s < shots; s++) {
        const double target = oracle_shot_draw(seed, s) * acc;
        uint64_t lo = 0, hi = N - 1;   /* smallest x with cum[x] > target */
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (cum[mid] > target) hi = mid; else lo = mid + 1;
        }
        out[s] = og_pack_bits(lo, mask);
    }
    free(cum);
    return 0;
}

/* -------------------------------------------------------- measurement -- */

void oracle_prob(const double *psi, int n, int q, double *p0, double *p1)
{
    const cd *a = (const cd *)psi;
    const uint64_t N = (uint64_t)1 << n;
    double s0 = 0, s1 = 0;
    for (uint64_t i = 0; i < N; i++) {
        double w = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
        if ((i >> q) & 1) s1 += w; else s0 += w;
    }
    *p0 = s0;
    *p1 = s1;
}

static void og_collapse(cd *a, int n, int q, int outcome, double p_out)
{
    const uint64_t N = (uint64_t)1 << n;
    const double scale = 1.0 / sqrt(p_out);
    for (uint64_t i = 0; i < N; i++) {
        if ((int)((i >> q) & 1) == outcome) a[i] = a[i] * scale;
        else a[i] = 0;
    }
}

/*
 * One measurement of qubit q with draw ordinal k.
 * mode 0: outcome 0 iff u(seed,k) < p0/(p0+p1); mode 1 (assertion): outcome 0
 * if p0/(p0+p1) > thr, else OG_E_ZEROPROB with the state left unchanged.
 * *prob receives the normalised probability of the recorded outcome.
 */
int oracle_measure(double *psi, int n, int q, uint64_t seed, uint64_t k, int mode,
                   double thr, int *outcome, double *prob)
{
    double p0, p1;
    oracle_prob(psi, n, q, &p0, &p1);
    double tot = p0 + p1;
    double P0 = p0 / tot;
    int out;
    if (mode & OG_MEAS_ASSERT) {
        if (!(P0 > thr)) {
            *outcome = -1;
            *prob = P0;
            return OG_E_ZEROPROB;
        }
        out = 0;
    } else {
        double u = oracle_draw(seed, k);
        out = (u < P0) ? 0 : 1;
    }
    og_collapse((cd *)psi, n, q, out, out == 0 ? p0 : p1);
    *outcome = out;
    *prob = out == 0 ? P0 : p1 / tot;
    return OG_OK;
}

/* reset: a drawn measurement followed by moving the |1> half onto |0>. */
int oracle_reset(double *psi, int n, int q, uint64_t seed, uint64_t k, int *outcome, double *prob)
{
    int st = oracle_measure(psi, n, q, seed, k, 0, 0.0, outcome, prob);
    if (st != OG_OK) return st;
    if (*outcome == 1) {
        cd *a = (cd *)psi;
        const uint64_t N = (uint64_t)1 << n, bq = (uint64_t)1 << q;
        for (uint64_t i = 0; i < N; i++) {
            if (i & bq) {
                a[i & ~bq] = a[i];
                a[i] = 0;
            }
        }
    }
    return OG_OK;
}

/* ------------------------------------------------------- circuit driver -- */

/*
 * Apply G gate records in order to psi (2^n interleaved complex doubles),
 * unfused: every gate by Eq. (1q-op) or Eq. (2q-op).  MEASURE and RESET use
 * draw ordinal *ordinal and then increment it; each appends (outcome, prob) to
 * the log while there is room (cap records).  BARRIER does nothing here.
 * Returns OG_OK, OG_E_INVAL (bad record: processing stops before it) or
 * OG_E_ZEROPROB (failed assertion: processing stops, state as before it).
 */
int oracle_run(double *psi, int n, const og_gate *g, size_t G, const double *mats,
               uint64_t seed, uint64_t *ordinal, double thr,
               int32_t *outcomes, double *probs, size_t cap, size_t *n_log)
{
    cd *a = (cd *)psi;
    double mbuf[32];
    cd m[16];
    size_t logged = n_log ? *n_log : 0;
    for (size_t i = 0; i < G; i++) {
        const og_gate *x = &g[i];
        int op = x->op;
        if (og_is_1q(op)) {
            if (x->q0 >= (uint32_t)n) return OG_E_INVAL;
            if (oracle_gate_matrix(x, mats, mbuf) != 2) return OG_E_INVAL;
            for (int j = 0; j < 4; j++) m[j] = mbuf[2 * j] + I * mbuf[2 * j + 1];
            og_apply_1q(a, n, (int)x->q0, m);
        } else if (og_is_2q(op)) {
            if (x->q0 >= (uint32_t)n || x->q1 >= (uint32_t)n || x->q0 == x->q1) return OG_E_INVAL;
            if (oracle_gate_matrix(x, mats, mbuf) != 4) return OG_E_INVAL;
            for (int j = 0; j < 16; j++) m[j] = mbuf[2 * j] + I * mbuf[2 * j + 1];
            og_apply_2q(a, n, (int)x->q0, (int)x->q1, m);
        } else if (op == OG_MEASURE || op == OG_RESET) {
            if (x->q0 >= (uint32_t)n) return OG_E_INVAL;
            int out;
            double pr;
            int st = (op == OG_MEASURE)
                ? oracle_measure(psi, n, (int)x->q0, seed, *ordinal, x->flags & OG_MEAS_ASSERT, thr, &out, &pr)
                : oracle_reset(psi, n, (int)x->q0, seed, *ordinal, &out, &pr);
            if (logged < cap) {
                outcomes[logged] = out;
                probs[logged] = pr;
            }
            logged++;
            if (n_log) *n_log = logged;
            if (st != OG_OK) return st;
            *ordinal += 1;
        } else if (op == OG_BARRIER) {
            continue;
        } else {
            return OG_E_INVAL;
        }
    }
    return OG_OK;
}

/* ------------------------------------------------------- expectation -- */

/*
 * out[t] = coef_t * Re <psi| P_t |psi>, P_t = (x) over qubits of X, Y or Z.
 * Written from the matrix entries: P_t |j> = i^{#Y} (-1)^{popcount(j & z)} |j ^ x>,
 * so <psi|P|psi> = sum_j conj(a_{j^x}) i^{#Y} (-1)^{popcount(j&z)} a_j.
 */
void oracle_expect(const double *psi, int n, const og_term *t, size_t T, double *out)
{
    const cd *a = (const cd *)psi;
    const uint64_t N = (uint64_t)1 << n;
    for (size_t k = 0; k < T; k++) {
        uint64_t x = t[k].x, z = t[k].z;
        int ny = __builtin_popcountll(x & z);
        cd iy = 1;
        for (int j = 0; j < (ny & 3); j++) iy *= I;
        cd acc = 0;
        for (uint64_t j = 0; j < N; j++) {
            double sign = (__builtin_popcountll(j & z) & 1) ? -1.0 : 1.0;
            acc += conj(a[j ^ x]) * iy * sign * a[j];
        }
        out[k] = t[k].coef * creal(acc);
    }
}
