/*
 * FP64 state-vector simulator: the plain definition of the amplitudes
 * <x|C|0^n> (Sec. "Multi-batch simulator", the amplitude of bitstring s_i of
 * circuit C) and of the linear XEB  F = 2^n/k * sum_i p_C(s_i) - 1 (Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the CPU oracle that checks
 * the CUDA path; the library never links, loads or calls it.
 *
 * Conventions: the state psi has 2^n complex128 entries stored as interleaved
 * (re, im) doubles; basis index x has bit q = qubit q.  A 1-qubit gate is a
 * 2x2 matrix acting as out = M in.  A 2-qubit gate on (qa, qb) is a 4x4 matrix
 * in the basis |b_a b_b> (qa's bit is the high bit).  Gates are applied one at
 * a time, in time order, with no fusion and no reordering.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}
static inline cplx cadd(cplx a, cplx b) {
    cplx r = { a.re + b.re, a.im + b.im };
    return r;
}

/* psi := |0...0> */
void sv_init_zero(double* psi, int n) {
    size_t dim = (size_t)1 << n;
    memset(psi, 0, dim * 2 * sizeof(double));
    psi[0] = 1.0;
}

/* Apply a 1-qubit gate m (2x2, row-major, interleaved complex) on qubit q. */
void sv_apply_1q(double* psi_d, int n, int q, const double* m_d) {
    cplx* psi = (cplx*)psi_d;
    const cplx* m = (const cplx*)m_d;
    size_t half = (size_t)1 << (n - 1);
    size_t low_mask = ((size_t)1 << q) - 1;
    long long h;
#pragma omp parallel for schedule(static)
    for (h = 0; h < (long long)half; ++h) {
        /* insert a 0 bit at position q */
        size_t x0 = (((size_t)h & ~low_mask) << 1) | ((size_t)h & low_mask);
        size_t x1 = x0 | ((size_t)1 << q);
        cplx a0 = psi[x0], a1 = psi[x1];
        psi[x0] = cadd(cmul(m[0], a0), cmul(m[1], a1));
        psi[x1] = cadd(cmul(m[2], a0), cmul(m[3], a1));
    }
}

/* Apply a 2-qubit gate m (4x4, row-major, interleaved complex) on (qa, qb). */
void sv_apply_2q(double* psi_d, int n, int qa, int qb, const double* m_d) {
    cplx* psi = (cplx*)psi_d;
    const cplx* m = (const cplx*)m_d;
    int lo = qa < qb ? qa : qb, hi = qa < qb ? qb : qa;
    size_t quarter = (size_t)1 << (n - 2);
    size_t lo_mask = ((size_t)1 << lo) - 1;
    size_t hi_mask = ((size_t)1 << hi) - 1;
    size_t ba = (size_t)1 << qa, bb = (size_t)1 << qb;
    long long h;
#pragma omp parallel for schedule(static)
    for (h = 0; h < (long long)quarter; ++h) {
        /* insert 0 bits at positions lo then hi */
        size_t t = (((size_t)h & ~lo_mask) << 1) | ((size_t)h & lo_mask);
        size_t base = ((t & ~hi_mask) << 1) | (t & hi_mask);
        size_t idx[4];
        cplx in[4];
        int r, c;
        /* basis order |b_a b_b>: index 2*b_a + b_b */
        idx[0] = base;
        idx[1] = base | bb;
        idx[2] = base | ba;
        idx[3] = base | ba | bb;
        for (c = 0; c < 4; ++c) in[c] = psi[idx[c]];
        for (r = 0; r < 4; ++r) {
            cplx acc = { 0.0, 0.0 };
            for (c = 0; c < 4; ++c) acc = cadd(acc, cmul(m[4 * r + c], in[c]));
            psi[idx[r]] = acc;
        }
    }
}

/* Run a whole circuit from |0^n>.  kinds[g] = 1 (1-qubit) or 2 (2-qubit);
 * mats is (n_gates, 4, 4) interleaved complex; a 1-qubit gate uses its
 * top-left 2x2 block. */
void sv_run_circuit(double* psi, int n, int n_gates, const int32_t* kinds,
                    const int32_t* q0, const int32_t* q1, const double* mats) {
    int g;
    sv_init_zero(psi, n);
    for (g = 0; g < n_gates; ++g) {
        const double* m = mats + (size_t)g * 32;
        if (kinds[g] == 1) {
            double m2[8];
            m2[0] = m[0]; m2[1] = m[1]; m2[2] = m[2]; m2[3] = m[3];
            m2[4] = m[8]; m2[5] = m[9]; m2[6] = m[10]; m2[7] = m[11];
            sv_apply_1q(psi, n, q0[g], m2);
        } else {
            sv_apply_2q(psi, n, q0[g], q1[g], m);
        }
    }
}

/* out[i] = psi[x_i] (interleaved complex) */
void sv_gather(const double* psi, size_t k, const uint64_t* x, double* out) {
    size_t i;
    for (i = 0; i < k; ++i) {
        out[2 * i] = psi[2 * x[i]];
        out[2 * i + 1] = psi[2 * x[i] + 1];
    }
}

/* sum_x |psi_x|^2 and sum_x |psi_x|^4 (norm and collision probability). */
void sv_moments(const double* psi_d, int n, double* s2, double* s4) {
    size_t dim = (size_t)1 << n;
    double a = 0.0, b = 0.0;
    long long x;
#pragma omp parallel for reduction(+ : a, b) schedule(static)
    for (x = 0; x < (long long)dim; ++x) {
        double p = psi_d[2 * x] * psi_d[2 * x] + psi_d[2 * x + 1] * psi_d[2 * x + 1];
        a += p;
        b += p * p;
    }
    *s2 = a;
    *s4 = b;
}

/* Inverse-CDF sampling of x ~ |psi_x|^2: for each u_j in [0,1) (sorted
 * ascending by the caller), out[j] = smallest x with cdf(x) > u_j * total. */
void sv_sample_sorted(const double* psi_d, int n, size_t m, const double* u_sorted,
                      uint64_t* out) {
    size_t dim = (size_t)1 << n, x = 0, j = 0;
    double total = 0.0, cdf = 0.0;
    for (x = 0; x < dim; ++x)
        total += psi_d[2 * x] * psi_d[2 * x] + psi_d[2 * x + 1] * psi_d[2 * x + 1];
    x = 0;
    cdf = psi_d[0] * psi_d[0] + psi_d[1] * psi_d[1];
    for (j = 0; j < m; ++j) {
        double target = u_sorted[j] * total;
        while (cdf <= target && x + 1 < dim) {
            ++x;
            cdf += psi_d[2 * x] * psi_d[2 * x] + psi_d[2 * x + 1] * psi_d[2 * x + 1];
        }
        out[j] = (uint64_t)x;
    }
}
