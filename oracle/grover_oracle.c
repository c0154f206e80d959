/*
 * grover_oracle.c -- plain, slow FP64 CPU oracle for the Grover iterator.
 *
 * TEST INFRASTRUCTURE ONLY (see grover_oracle.h).  Straight loops in index
 * order, no blocking, no fusion, no threads: each function is meant to be
 * checked against the paper by eye.
 *
 * Readings of the paper taken here (where its listings are garbled):
 *   - loops over basis states cover all N indices (the printed bound N-1 would
 *     leave the last amplitude untouched and break norm preservation);
 *   - the inversion about the mean is unconditional over all amplitudes (the
 *     printed test compares an amplitude with a ket and has no meaning); its
 *     divisor is N = 2^n;
 *   - the single-qubit gate is the out-of-place pair butterfly of Eq.
 *     (unitary) (the listing's "+=" into psi would double count);
 *   - the conditional phase shift is 2|0><0| - I exactly as written (keep c_0,
 *     negate the rest), so the circuit equals the operator form with no global
 *     phase.
 */
#include "grover_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int g_mutation = 0;

int or_set_mutation(int which) {
    int old = g_mutation;
    g_mutation = which;
    return old;
}

static uint64_t dim(int n) { return (uint64_t)1 << n; }

/* ---------------------------------------------------------------------- */
/* Neumaier's improved Kahan summation (A. Neumaier, ZAMM 54, 1974).        */
double or_neumaier_sum(const double *x, size_t count, size_t stride) {
    double sum = 0.0, comp = 0.0;
    for (size_t i = 0; i < count; ++i) {
        double v = x[i * stride];
        double t = sum + v;
        if (fabs(sum) >= fabs(v))
            comp += (sum - t) + v;
        else
            comp += (v - t) + sum;
        sum = t;
    }
    return sum + comp;
}

/* ---------------------------------------------------------------------- */
void or_init_zero(double *psi, int n) {
    memset(psi, 0, sizeof(double) * 2 * dim(n));
    psi[0] = 1.0;
}

void or_init_uniform(double *psi, int n) {
    uint64_t N = dim(n);
    double a = 1.0 / sqrt((double)N);
    for (uint64_t i = 0; i < N; ++i) {
        psi[2 * i] = a;
        psi[2 * i + 1] = 0.0;
    }
}

/* ---------------------------------------------------------------------- */
/* Algorithm "n-qubit Oracle": for each solution state k[i], psi[k[i]] *= -1. */
void or_oracle_list(double *psi, int n, const uint64_t *marked, size_t m) {
    (void)n;
    for (size_t i = 0; i < m; ++i) {
        uint64_t x = marked[i];
        if (g_mutation == 4) x = (x + 1) & (dim(n) - 1);
        psi[2 * x] = -psi[2 * x];
        psi[2 * x + 1] = -psi[2 * x + 1];
    }
}

void or_oracle_bitmask(double *psi, int n, const uint32_t *words) {
    uint64_t N = dim(n);
    for (uint64_t x = 0; x < N; ++x) {
        if ((words[x >> 5] >> (x & 31)) & 1u) {
            psi[2 * x] = -psi[2 * x];
            psi[2 * x + 1] = -psi[2 * x + 1];
        }
    }
}

/* Section "Inversion About Mean Operator": <c> = (1/N) sum_x c_x, the real and
 * imaginary sums kept separately as in Algorithm "n-qubit Inversion about
 * Mean". */
void or_mean(const double *psi, int n, double *mu_re, double *mu_im) {
    uint64_t N = dim(n);
    uint64_t count = (g_mutation == 1) ? N - 1 : N;
    double re = or_neumaier_sum(psi, count, 2);
    double im = or_neumaier_sum(psi + 1, count, 2);
    double div = (g_mutation == 8) ? (double)(N - 1) : (double)N;
    *mu_re = re / div;
    *mu_im = im / div;
}

/* Algorithm "n-qubit Inversion about Mean": the action of
 * Delta = 2|psi><psi| - I on sum_x c_x|x> is c_x -> 2<c> - c_x. */
void or_inversion_mean(double *psi, int n) {
    uint64_t N = dim(n);
    double mu_re, mu_im;
    or_mean(psi, n, &mu_re, &mu_im);
    double two_re = 2.0 * mu_re, two_im = 2.0 * mu_im;
    if (g_mutation == 3) {
        two_re = mu_re;
        two_im = mu_im;
    }
    uint64_t count = (g_mutation == 1) ? N - 1 : N;
    for (uint64_t x = 0; x < count; ++x) {
        psi[2 * x] = two_re - psi[2 * x];
        if (g_mutation == 5)
            psi[2 * x + 1] = psi[2 * x + 1] - two_im;
        else
            psi[2 * x + 1] = two_im - psi[2 * x + 1];
    }
}

/* Proposed grover_search: each iteration is oracle() then inversion_mean(). */
void or_grover_operator(double *psi, int n, const uint64_t *marked, size_t m,
                        uint64_t k) {
    for (uint64_t it = 0; it < k; ++it) {
        or_oracle_list(psi, n, marked, m);
        or_inversion_mean(psi, n);
    }
}

void or_grover_operator_bitmask(double *psi, int n, const uint32_t *words,
                                uint64_t k) {
    for (uint64_t it = 0; it < k; ++it) {
        or_oracle_bitmask(psi, n, words);
        or_inversion_mean(psi, n);
    }
}

/* ---------------------------------------------------------------------- */
/* Eq. (unitary) with U = H = (1/sqrt2)[[1,1],[1,-1]] on target qubit q: the
 * amplitudes of x (bit q = 0) and x|2^q (bit q = 1) become
 * (a + b)/sqrt2 and (a - b)/sqrt2. */
void or_hadamard_qubit(double *psi, int n, int q) {
    uint64_t N = dim(n);
    uint64_t s = (uint64_t)1 << q;
    const double r = 0.70710678118654752440; /* 1/sqrt(2) */
    for (uint64_t x = 0; x < N; ++x) {
        if (x & s) continue;
        uint64_t y = x | s;
        for (int c = 0; c < 2; ++c) {
            double a = psi[2 * x + c], b = psi[2 * y + c];
            double lo = (a + b) * r, hi = (a - b) * r;
            if (g_mutation == 6) {
                double t = lo;
                lo = hi;
                hi = t;
            }
            psi[2 * x + c] = lo;
            psi[2 * y + c] = hi;
        }
    }
}

void or_hadamard_all(double *psi, int n) {
    for (int q = 0; q < n; ++q) or_hadamard_qubit(psi, n, q);
}

/* Section "Background", stage 4: 2|0><0| - I flips every state except |0>. */
void or_phase_shift_zero(double *psi, int n) {
    uint64_t N = dim(n);
    if (g_mutation == 2) { /* I - 2|0><0| */
        psi[0] = -psi[0];
        psi[1] = -psi[1];
        return;
    }
    for (uint64_t x = 1; x < N; ++x) {
        psi[2 * x] = -psi[2 * x];
        psi[2 * x + 1] = -psi[2 * x + 1];
    }
}

/* Conventional grover_search: oracle, H^{(x)n}, 2|0><0|-I, H^{(x)n}. */
/* Pauli X on qubit q: the amplitudes of x and x ^ 2^q trade places. */
void or_x_qubit(double *psi, int n, int q) {
    uint64_t N = dim(n);
    uint64_t s = (uint64_t)1 << q;
    for (uint64_t x = 0; x < N; ++x) {
        if (x & s) continue;
        uint64_t y = x | s;
        for (int c = 0; c < 2; ++c) {
            double t = psi[2 * x + c];
            psi[2 * x + c] = psi[2 * y + c];
            psi[2 * y + c] = t;
        }
    }
}

/* Multi-controlled Z on all n qubits: phase -1 on |1...1>, visiting every
 * amplitude as a gate-level simulator does (one O(N) pass); negate_all also
 * multiplies the whole state by -1. */
void or_mcz(double *psi, int n, int negate_all) {
    uint64_t N = dim(n);
    for (uint64_t x = 0; x < N; ++x) {
        int flip = (x == N - 1);
        if (negate_all) flip = !flip;
        if (flip) {
            psi[2 * x] = -psi[2 * x];
            psi[2 * x + 1] = -psi[2 * x + 1];
        }
    }
}

uint64_t or_grover_circuit(double *psi, int n, const uint64_t *marked, size_t m, uint64_t k) {
    uint64_t gates = 0;
    for (uint64_t it = 0; it < k; ++it) {
        /* oracle, Fig. oracle1: X on each qubit where the solution has a 0,
         * the multi-controlled gate, the same X gates again */
        for (size_t i = 0; i < m; ++i) {
            for (int q = 0; q < n; ++q)
                if (!((marked[i] >> q) & 1)) { or_x_qubit(psi, n, q); ++gates; }
            or_mcz(psi, n, 0);
            ++gates;
            for (int q = 0; q < n; ++q)
                if (!((marked[i] >> q) & 1)) { or_x_qubit(psi, n, q); ++gates; }
        }
        for (int q = 0; q < n; ++q) { or_hadamard_qubit(psi, n, q); ++gates; }
        /* 2|0><0| - I = -X^{(x)n} (I - 2|1...1><1...1|) X^{(x)n} */
        for (int q = 0; q < n; ++q) { or_x_qubit(psi, n, q); ++gates; }
        or_mcz(psi, n, 1);
        ++gates;
        for (int q = 0; q < n; ++q) { or_x_qubit(psi, n, q); ++gates; }
        for (int q = 0; q < n; ++q) { or_hadamard_qubit(psi, n, q); ++gates; }
    }
    return gates;
}

void or_grover_gate(double *psi, int n, const uint64_t *marked, size_t m,
                    uint64_t k) {
    for (uint64_t it = 0; it < k; ++it) {
        or_oracle_list(psi, n, marked, m);
        or_hadamard_all(psi, n);
        or_phase_shift_zero(psi, n);
        or_hadamard_all(psi, n);
    }
}

/* ---------------------------------------------------------------------- */
uint64_t or_optimal_iterations(int n, uint64_t m) {
    if (m == 0) return 0;
    double r = sqrt((double)dim(n) / (double)m);
    return (uint64_t)floor(0.78539816339744830962 * r);
}

static double grover_theta(uint64_t N, uint64_t M) {
    /* sin(theta) = sqrt(M/N), cos(theta) = sqrt((N-M)/N) */
    return atan2(sqrt((double)M), sqrt((double)(N - M)));
}

void or_closed_form_uniform(int n, uint64_t m, uint64_t k, double *a_marked,
                            double *a_unmarked) {
    uint64_t N = dim(n);
    double th = grover_theta(N, m);
    double ang = (double)(2 * k + 1) * th;
    *a_marked = (m > 0) ? sin(ang) / sqrt((double)m) : 0.0;
    *a_unmarked = (m < N) ? cos(ang) / sqrt((double)(N - m)) : 0.0;
}

void or_closed_form_general(double *psi, int n, const uint64_t *marked,
                            size_t m, uint64_t k) {
    uint64_t N = dim(n);
    /* group sums in index order, compensated */
    double sm_re = 0, sm_im = 0, cm_re = 0, cm_im = 0; /* marked */
    double su_re = 0, su_im = 0, cu_re = 0, cu_im = 0; /* unmarked */
    size_t p = 0;
    for (uint64_t x = 0; x < N; ++x) {
        int is_m = (p < m && marked[p] == x);
        if (is_m) ++p;
        double v[2] = {psi[2 * x], psi[2 * x + 1]};
        double *s[2] = {is_m ? &sm_re : &su_re, is_m ? &sm_im : &su_im};
        double *c[2] = {is_m ? &cm_re : &cu_re, is_m ? &cm_im : &cu_im};
        for (int j = 0; j < 2; ++j) {
            double t = *s[j] + v[j];
            if (fabs(*s[j]) >= fabs(v[j]))
                *c[j] += (*s[j] - t) + v[j];
            else
                *c[j] += (v[j] - t) + *s[j];
            *s[j] = t;
        }
    }
    double M = (double)m, U = (double)(N - m);
    double al_re = (m > 0) ? (sm_re + cm_re) / M : 0.0;
    double al_im = (m > 0) ? (sm_im + cm_im) / M : 0.0;
    double be_re = (m < N) ? (su_re + cu_re) / U : 0.0;
    double be_im = (m < N) ? (su_im + cu_im) / U : 0.0;
    /* scaled coordinates u = sqrt(M) alpha, v = sqrt(N-M) beta */
    double u_re = sqrt(M) * al_re, u_im = sqrt(M) * al_im;
    double v_re = sqrt(U) * be_re, v_im = sqrt(U) * be_im;
    double ang = 2.0 * (double)k * grover_theta(N, m);
    if (g_mutation == 7) ang = -ang;
    double cs = cos(ang), sn = sin(ang);
    double uk_re = cs * u_re + sn * v_re, uk_im = cs * u_im + sn * v_im;
    double vk_re = -sn * u_re + cs * v_re, vk_im = -sn * u_im + cs * v_im;
    double ak_re = (m > 0) ? uk_re / sqrt(M) : 0.0;
    double ak_im = (m > 0) ? uk_im / sqrt(M) : 0.0;
    double bk_re = (m < N) ? vk_re / sqrt(U) : 0.0;
    double bk_im = (m < N) ? vk_im / sqrt(U) : 0.0;
    double esign = (k & 1) ? -1.0 : 1.0;
    p = 0;
    for (uint64_t x = 0; x < N; ++x) {
        if (p < m && marked[p] == x) {
            ++p;
            psi[2 * x] = ak_re + (psi[2 * x] - al_re);
            psi[2 * x + 1] = ak_im + (psi[2 * x + 1] - al_im);
        } else {
            psi[2 * x] = bk_re + esign * (psi[2 * x] - be_re);
            psi[2 * x + 1] = bk_im + esign * (psi[2 * x + 1] - be_im);
        }
    }
}

/* ---------------------------------------------------------------------- */
void or_probs(const double *psi, int n, double *p) {
    uint64_t N = dim(n);
    for (uint64_t x = 0; x < N; ++x)
        p[x] = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
}

double or_norm(const double *psi, int n) {
    uint64_t N = dim(n);
    double *p = (double *)malloc(sizeof(double) * N);
    if (!p) return NAN;
    or_probs(psi, n, p);
    double s = or_neumaier_sum(p, N, 1);
    free(p);
    return s;
}

double or_success_prob(const double *psi, int n, const uint64_t *marked,
                       size_t m) {
    (void)n;
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < m; ++i) {
        uint64_t x = marked[i];
        double v = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
        double t = s + v;
        if (fabs(s) >= fabs(v))
            c += (s - t) + v;
        else
            c += (v - t) + s;
        s = t;
    }
    return s + c;
}

/* (p desc, index asc): the m best kept in a sorted array, one scan. */
void or_topm(const double *psi, int n, size_t m, uint64_t *idx, double *p) {
    uint64_t N = dim(n);
    size_t have = 0;
    for (uint64_t x = 0; x < N; ++x) {
        double v = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
        /* an equal probability never displaces a lower index seen earlier */
        if (have == m && !(v > p[m - 1])) continue;
        size_t pos = (have < m) ? have : m - 1;
        while (pos > 0 && v > p[pos - 1]) {
            p[pos] = p[pos - 1];
            idx[pos] = idx[pos - 1];
            --pos;
        }
        p[pos] = v;
        idx[pos] = x;
        if (have < m) ++have;
    }
}

/* ---------------------------------------------------------------------- */
/* Generalised phase iterator: O(phi) multiplies the marked amplitudes by
 * e^{i phi}; D(vphi) = I + (e^{i vphi} - 1)|s><s|, i.e. c_i <- c_i -
 * (1 - e^{i vphi}) <c> with <c> the complex mean. */
void or_phase_grover(double *psi, int n, const uint64_t *marked, size_t m, const double *phi,
                     const double *vphi, uint64_t K) {
    uint64_t N = dim(n);
    for (uint64_t t = 0; t < K; ++t) {
        double cr = cos(phi[t]), sr = sin(phi[t]);
        for (size_t i = 0; i < m; ++i) {
            uint64_t x = marked[i];
            double re = psi[2 * x], im = psi[2 * x + 1];
            psi[2 * x] = cr * re - sr * im;
            psi[2 * x + 1] = sr * re + cr * im;
        }
        double mu_re, mu_im;
        or_mean(psi, n, &mu_re, &mu_im);
        /* kappa = (1 - e^{i vphi}) mu */
        double ar = 1.0 - cos(vphi[t]), ai = -sin(vphi[t]);
        double kr = ar * mu_re - ai * mu_im, ki = ar * mu_im + ai * mu_re;
        for (uint64_t x = 0; x < N; ++x) {
            psi[2 * x] -= kr;
            psi[2 * x + 1] -= ki;
        }
    }
}

double or_phase_loss(const double *psi, int n, const uint64_t *marked, size_t m) {
    return -log(or_success_prob(psi, n, marked, m));
}

double or_phase_reduced(int n, uint64_t m, const double *phi, const double *vphi, uint64_t K,
                        double *alpha_re, double *alpha_im, double *beta_re, double *beta_im) {
    double N = (double)dim(n), M = (double)m;
    double a0 = 1.0 / sqrt(N);
    double ar = a0, ai = 0.0, br = a0, bi = 0.0;
    for (uint64_t t = 0; t < K; ++t) {
        double cr = cos(phi[t]), sr = sin(phi[t]);
        double nr = cr * ar - sr * ai, ni = sr * ar + cr * ai;
        ar = nr;
        ai = ni;
        double mu_re = (M * ar + (N - M) * br) / N, mu_im = (M * ai + (N - M) * bi) / N;
        double qr = 1.0 - cos(vphi[t]), qi = -sin(vphi[t]);
        double kr = qr * mu_re - qi * mu_im, ki = qr * mu_im + qi * mu_re;
        ar -= kr;
        ai -= ki;
        br -= kr;
        bi -= ki;
    }
    *alpha_re = ar;
    *alpha_im = ai;
    *beta_re = br;
    *beta_im = bi;
    return -log(M * (ar * ar + ai * ai));
}
