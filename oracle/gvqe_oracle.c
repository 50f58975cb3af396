/*
 * gvqe_oracle.c -- plain, slow, obviously correct CPU oracle for the
 * Graph-VQE energy / gradient path (arxiv 2607.02749).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (all in complex128, accumulation in double):
 *   - the ansatz state |psi(theta)> = U(theta)|0...0> of Section IV-B: an
 *     initial rotation layer followed by D repetitions of [CNOT entangler,
 *     rotation layer] (Eq. 7 gate matrix, Eq. 8 parameter count); a rotation
 *     layer is RY on every qubit (flattened index p = r*n + q) or, with gate
 *     set 2, the full EfficientSU2 layer RY then RZ on every qubit;
 *   - the Pauli-sum Hamiltonian applied term by term, H = sum_k c_k P_k
 *     (Eq. 6), each P_k applied letter by letter with the standard matrices;
 *   - the energy E = <psi|H|psi> (Eq. 4);
 *   - dE/dtheta by a gate-by-gate adjoint (reverse) sweep, and by the
 *     parameter-shift rule of Eq. 13.
 *
 * Conventions (readings where the paper is silent): qubit q is bit q of the
 * basis index x; character i of a Pauli string acts on qubit i; the linear
 * entangler is CX(0,1), CX(1,2), ..., CX(n-2,n-1) applied in that order (the
 * other entanglers are listed at entangler_gates below).
 *
 * Every gate is applied one at a time in circuit order; there is no fusion,
 * no table, no Walsh-Hadamard transform and no grouping of terms.
 *
 * Return codes: 0 ok, -1 invalid argument, -2 out of memory.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* Largest register the oracle accepts (a 2^30 complex128 state is 16 GiB). */
#define ORACLE_MAX_QUBITS 30

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- gates -- */

/* RY(theta) on qubit q, Eq. 7: [[cos t/2, -sin t/2], [sin t/2, cos t/2]]. */
static void apply_ry(cplx *psi, int n, int q, double theta) {
    const double c = cos(0.5 * theta), s = sin(0.5 * theta);
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        if (x & bit) continue;
        const cplx a = psi[x], b = psi[x | bit];
        psi[x] = c * a - s * b;
        psi[x | bit] = s * a + c * b;
    }
}

/* RZ(theta) on qubit q, the RZ of Eq. 7-8's EfficientSU2 layers:
 * diag(exp(-i theta/2), exp(+i theta/2)). */
static void apply_rz(cplx *psi, int n, int q, double theta) {
    const cplx p0 = cos(0.5 * theta) - I * sin(0.5 * theta);
    const cplx p1 = cos(0.5 * theta) + I * sin(0.5 * theta);
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; ++x) psi[x] *= (x & bit) ? p1 : p0;
}

/*
 * Gate set of a rotation layer.  1: RY on every qubit (P = n (D+1)).  2: the
 * full EfficientSU2 layer of Eq. 8, RY on every qubit and then RZ on every
 * qubit (P = 2 n (D+1)); layer r's RY angles are theta[2 r n + q] and its RZ
 * angles theta[2 r n + n + q].  A process-wide setting of this test oracle.
 */
static int g_gates = 1;

int oracle_set_gates(int gates) {
    if (gates != 1 && gates != 2) return ORACLE_EINVAL;
    g_gates = gates;
    return ORACLE_OK;
}

/* CNOT with control qubit `ctl` and target qubit `tgt`: |x> -> |x xor (x_ctl << tgt)>. */
static void apply_cx(cplx *psi, int n, int ctl, int tgt) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t cb = (int64_t)1 << ctl, tb = (int64_t)1 << tgt;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        if ((x & cb) && !(x & tb)) {
            const cplx t = psi[x];
            psi[x] = psi[x | tb];
            psi[x | tb] = t;
        }
    }
}

/*
 * Entanglers as ordered CNOT lists (control, target).  Section IV-B names
 * linear, circular and full; Section V-A and Table 2 add reverse linear,
 * pairwise and SCA (shifted-circular-alternating).  The paper prints none of
 * the orders; these are the readings used throughout:
 *   0 linear:         CX(0,1), CX(1,2), ..., CX(n-2,n-1)
 *   1 circular:       CX(n-1,0) (the wrap-around), then the linear list
 *   2 full:           CX(i,j) for every i < j, i ascending, j ascending within i
 *   3 reverse linear: CX(n-2,n-1), CX(n-3,n-2), ..., CX(0,1)
 *   4 pairwise:       CX(i,i+1) for even i ascending, then for odd i ascending
 *   5 SCA:            in entangler layer r (r = 1 .. reps, offset o = r - 1) the
 *                     circular list rotated right by o mod n (its last o gates
 *                     move to the front), with control and target swapped in
 *                     every gate when o is odd
 * The entangler in use is a process-wide setting of this test oracle.
 */
static int g_entangler = 0;

int oracle_set_entangler(int ent) {
    if (ent < 0 || ent > 5) return ORACLE_EINVAL;
    g_entangler = ent;
    return ORACLE_OK;
}

static int entangler_gates(int n, int layer, int *ctl, int *tgt) {
    int k = 0;
    if (g_entangler == 2) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                ctl[k] = i;
                tgt[k++] = j;
            }
        return k;
    }
    if (g_entangler == 3) {
        for (int q = n - 2; q >= 0; --q) {
            ctl[k] = q;
            tgt[k++] = q + 1;
        }
        return k;
    }
    if (g_entangler == 4) {
        for (int start = 0; start < 2; ++start)
            for (int q = start; q + 1 < n; q += 2) {
                ctl[k] = q;
                tgt[k++] = q + 1;
            }
        return k;
    }
    if ((g_entangler == 1 || g_entangler == 5) && n > 1) {
        ctl[k] = n - 1;
        tgt[k++] = 0;
    }
    for (int q = 0; q + 1 < n; ++q) {
        ctl[k] = q;
        tgt[k++] = q + 1;
    }
    if (g_entangler == 5 && k > 0) {
        /* rotate the circular list right by o, then swap roles for odd o */
        const int o = (layer - 1) % k;
        int c2[ORACLE_MAX_QUBITS], t2[ORACLE_MAX_QUBITS];
        for (int g = 0; g < k; ++g) {
            c2[(g + o) % k] = ctl[g];
            t2[(g + o) % k] = tgt[g];
        }
        const int swap = (layer - 1) & 1;
        for (int g = 0; g < k; ++g) {
            ctl[g] = swap ? t2[g] : c2[g];
            tgt[g] = swap ? c2[g] : t2[g];
        }
    }
    return k;
}

/* The entangler of layer r (r >= 1), one gate at a time in its order. */
static void apply_entangler(cplx *psi, int n, int layer) {
    int ctl[ORACLE_MAX_QUBITS * ORACLE_MAX_QUBITS], tgt[ORACLE_MAX_QUBITS * ORACLE_MAX_QUBITS];
    const int k = entangler_gates(n, layer, ctl, tgt);
    for (int g = 0; g < k; ++g) apply_cx(psi, n, ctl[g], tgt[g]);
}

/* Its inverse: the same CNOTs in reverse order (each is its own inverse). */
static void apply_entangler_inverse(cplx *psi, int n, int layer) {
    int ctl[ORACLE_MAX_QUBITS * ORACLE_MAX_QUBITS], tgt[ORACLE_MAX_QUBITS * ORACLE_MAX_QUBITS];
    const int k = entangler_gates(n, layer, ctl, tgt);
    for (int g = k - 1; g >= 0; --g) apply_cx(psi, n, ctl[g], tgt[g]);
}

/* U(theta)|0> for the RY+CX ansatz (Section IV-B, Eq. 7-8). */
/* Rotation layer r: RY on every qubit, then (gate set 2) RZ on every qubit. */
static void apply_rotation_layer(cplx *psi, int n, int r, const double *theta) {
    const int base = r * g_gates * n;
    for (int q = 0; q < n; ++q) apply_ry(psi, n, q, theta[base + q]);
    if (g_gates == 2)
        for (int q = 0; q < n; ++q) apply_rz(psi, n, q, theta[base + n + q]);
}

static void prepare_state(cplx *psi, int n, int reps, const double *theta) {
    const int64_t dim = (int64_t)1 << n;
    memset(psi, 0, sizeof(cplx) * (size_t)dim);
    psi[0] = 1.0;
    apply_rotation_layer(psi, n, 0, theta);
    for (int r = 1; r <= reps; ++r) {
        apply_entangler(psi, n, r);
        apply_rotation_layer(psi, n, r, theta);
    }
}

/* ---------------------------------------------------------- Hamiltonian -- */

/*
 * Apply one Pauli string P (letters over {I,X,Y,Z}, character i on qubit i)
 * with weight `coef`, accumulating out += coef * P psi.  Letters act as
 * X|b> = |1-b>, Y|b> = i(-1)^b |1-b>, Z|b> = (-1)^b |b>  (Eq. 6 operators).
 * The map x -> image(x) is a bijection, so the parallel loop has no conflicts.
 */
static int apply_pauli_term(cplx *out, const cplx *psi, int n, const char *str, double coef) {
    int qs[ORACLE_MAX_QUBITS];
    char ls[ORACLE_MAX_QUBITS];
    int w = 0;
    for (int q = 0; q < n; ++q) {
        const char L = str[q];
        if (L == 'I') continue;
        if (L != 'X' && L != 'Y' && L != 'Z') return ORACLE_EINVAL;
        qs[w] = q;
        ls[w] = L;
        ++w;
    }
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        int64_t y = x;
        cplx phase = 1.0;
        for (int j = 0; j < w; ++j) {
            const int64_t bit = (int64_t)1 << qs[j];
            const int b = (x & bit) ? 1 : 0;
            if (ls[j] == 'X') {
                y ^= bit;
            } else if (ls[j] == 'Y') {
                phase *= b ? -I : I;
                y ^= bit;
            } else { /* 'Z' */
                if (b) phase = -phase;
            }
        }
        out[y] += coef * phase * psi[x];
    }
    return ORACLE_OK;
}

/* out = H psi with H = sum_k c_k P_k (Eq. 6), term by term. */
static int apply_hamiltonian(cplx *out, const cplx *psi, int n, int n_terms,
                             const char *pauli, const double *coeffs) {
    const int64_t dim = (int64_t)1 << n;
    memset(out, 0, sizeof(cplx) * (size_t)dim);
    for (int k = 0; k < n_terms; ++k) {
        const int rc = apply_pauli_term(out, psi, n, pauli + (size_t)k * (size_t)n, coeffs[k]);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

/* <a|b> */
static cplx inner(const cplx *a, const cplx *b, int n) {
    const int64_t dim = (int64_t)1 << n;
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        const cplx t = conj(a[x]) * b[x];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

/* Im <lam| Y_q |psi>, with (Y psi)[x] = -i psi[x^bit] if x_q = 0 and +i psi[x^bit] if x_q = 1. */
static double im_lam_y_psi(const cplx *lam, const cplx *psi, int n, int q) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
    double acc = 0.0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        const cplx ypsi = (x & bit) ? I * psi[x ^ bit] : -I * psi[x ^ bit];
        acc += cimag(conj(lam[x]) * ypsi);
    }
    return acc;
}

/* Im <lam| Z_q |psi>, the RZ derivative 2 Re <lam| (-i/2) Z_q |psi>. */
static double im_lam_z_psi(const cplx *lam, const cplx *psi, int n, int q) {
    const int64_t dim = (int64_t)1 << n;
    const int64_t bit = (int64_t)1 << q;
    double acc = 0.0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        const cplx zpsi = (x & bit) ? -psi[x] : psi[x];
        acc += cimag(conj(lam[x]) * zpsi);
    }
    return acc;
}

static int check_args(int n, int reps) {
    if (n < 1 || n > ORACLE_MAX_QUBITS || reps < 0) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* ----------------------------------------------------------- public API -- */

/* psi_out: 2 * 2^n doubles, interleaved (re, im). */
int oracle_state(int n, int reps, const double *theta, double *psi_out) {
    if (check_args(n, reps) || !theta || !psi_out) return ORACLE_EINVAL;
    prepare_state((cplx *)psi_out, n, reps, theta);
    return ORACLE_OK;
}

/* out = H psi; psi and out are interleaved complex arrays of 2^n entries. */
int oracle_apply_hamiltonian(int n, int n_terms, const char *pauli, const double *coeffs,
                             const double *psi, double *out) {
    if (n < 1 || n > ORACLE_MAX_QUBITS || n_terms < 0 || !psi || !out) return ORACLE_EINVAL;
    if (n_terms > 0 && (!pauli || !coeffs)) return ORACLE_EINVAL;
    return apply_hamiltonian((cplx *)out, (const cplx *)psi, n, n_terms, pauli, coeffs);
}

/* E = <psi|H|psi> (Eq. 4), returned as the real part; *E_imag receives the
 * imaginary part (zero up to rounding for a Hermitian H) when non-NULL. */
int oracle_energy(int n, int reps, const double *theta, int n_terms, const char *pauli,
                  const double *coeffs, double *E, double *E_imag) {
    if (check_args(n, reps) || !theta || !E || n_terms < 0) return ORACLE_EINVAL;
    const size_t dim = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * dim);
    cplx *hpsi = (cplx *)malloc(sizeof(cplx) * dim);
    if (!psi || !hpsi) { free(psi); free(hpsi); return ORACLE_ENOMEM; }
    prepare_state(psi, n, reps, theta);
    int rc = apply_hamiltonian(hpsi, psi, n, n_terms, pauli, coeffs);
    if (!rc) {
        const cplx e = inner(psi, hpsi, n);
        *E = creal(e);
        if (E_imag) *E_imag = cimag(e);
    }
    free(psi);
    free(hpsi);
    return rc;
}

/*
 * Energy and its full gradient by the adjoint method: lam = H psi at the end of
 * the circuit, then the gates are walked in reverse order.  At each RY gate the
 * derivative is 2 Re <lam| dU/dtheta |psi> = Im <lam| Y_q |psi> (RY = exp(-i t Y/2)),
 * at each RZ gate Im <lam| Z_q |psi>, evaluated with psi and lam taken right
 * after that gate; then the gate's inverse is applied to both.  CNOTs are their
 * own inverse.
 */
int oracle_energy_grad(int n, int reps, const double *theta, int n_terms, const char *pauli,
                       const double *coeffs, double *E, double *grad) {
    if (check_args(n, reps) || !theta || !E || !grad || n_terms < 0) return ORACLE_EINVAL;
    const size_t dim = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * dim);
    cplx *lam = (cplx *)malloc(sizeof(cplx) * dim);
    if (!psi || !lam) { free(psi); free(lam); return ORACLE_ENOMEM; }
    prepare_state(psi, n, reps, theta);
    int rc = apply_hamiltonian(lam, psi, n, n_terms, pauli, coeffs);
    if (rc) { free(psi); free(lam); return rc; }
    *E = creal(inner(psi, lam, n));
    for (int r = reps; r >= 0; --r) {
        const int base = r * g_gates * n;
        if (g_gates == 2) {
            for (int q = n - 1; q >= 0; --q) {
                const int p = base + n + q;
                grad[p] = im_lam_z_psi(lam, psi, n, q);
                apply_rz(psi, n, q, -theta[p]);
                apply_rz(lam, n, q, -theta[p]);
            }
        }
        for (int q = n - 1; q >= 0; --q) {
            const int p = base + q;
            grad[p] = im_lam_y_psi(lam, psi, n, q);
            apply_ry(psi, n, q, -theta[p]);
            apply_ry(lam, n, q, -theta[p]);
        }
        if (r > 0) {
            apply_entangler_inverse(psi, n, r);
            apply_entangler_inverse(lam, n, r);
        }
    }
    free(psi);
    free(lam);
    return ORACLE_OK;
}

/*
 * Parameter-shift gradient, Eq. 13:
 *   dE/dtheta_p = 1/2 [E(theta + pi/2 e_p) - E(theta - pi/2 e_p)].
 * Entries with mask[p] == 0 are set to 0 (mask may be NULL = all active).
 */
int oracle_param_shift_grad(int n, int reps, const double *theta, int n_terms,
                            const char *pauli, const double *coeffs,
                            const unsigned char *mask, double *grad) {
    if (check_args(n, reps) || !theta || !grad || n_terms < 0) return ORACLE_EINVAL;
    const int P = g_gates * n * (reps + 1);
    double *shifted = (double *)malloc(sizeof(double) * (size_t)P);
    if (!shifted) return ORACLE_ENOMEM;
    const double half_pi = 2.0 * atan(1.0);
    int rc = ORACLE_OK;
    for (int p = 0; p < P && !rc; ++p) {
        if (mask && !mask[p]) { grad[p] = 0.0; continue; }
        double ep, em;
        memcpy(shifted, theta, sizeof(double) * (size_t)P);
        shifted[p] = theta[p] + half_pi;
        rc = oracle_energy(n, reps, shifted, n_terms, pauli, coeffs, &ep, NULL);
        if (rc) break;
        shifted[p] = theta[p] - half_pi;
        rc = oracle_energy(n, reps, shifted, n_terms, pauli, coeffs, &em, NULL);
        if (rc) break;
        grad[p] = 0.5 * (ep - em);
    }
    free(shifted);
    return rc;
}

/*
 * Bounded-work timing helper for the CPU baseline: applies the first
 * `n_gates` RY gates of the circuit's first layer to a fresh |0> state and the
 * first `n_terms` Pauli terms once, so a caller can time a measured fraction
 * of one evaluation and scale it.  Returns 0 on success.
 */
int oracle_partial_work(int n, int n_gates, int n_terms, const char *pauli,
                        const double *coeffs, const double *theta, double *checksum) {
    if (n < 1 || n > ORACLE_MAX_QUBITS || n_gates < 0 || n_terms < 0 || !checksum) return ORACLE_EINVAL;
    const size_t dim = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * dim);
    cplx *out = (cplx *)malloc(sizeof(cplx) * dim);
    if (!psi || !out) { free(psi); free(out); return ORACLE_ENOMEM; }
    memset(psi, 0, sizeof(cplx) * dim);
    memset(out, 0, sizeof(cplx) * dim);
    psi[0] = 1.0;
    for (int g = 0; g < n_gates; ++g) apply_ry(psi, n, g % n, theta[g]);
    int rc = ORACLE_OK;
    for (int k = 0; k < n_terms && !rc; ++k)
        rc = apply_pauli_term(out, psi, n, pauli + (size_t)k * (size_t)n, coeffs[k]);
    if (!rc) *checksum = creal(inner(psi, out, n));
    free(psi);
    free(out);
    return rc;
}

/*
 * Timing helper for the CPU baseline: on one 2^n state, times `n_gates` RY
 * sweeps (apply_ry) and `n_terms` Pauli-term sweeps (apply_pauli_term) of the
 * oracle separately, excluding allocation.  Writes seconds per sweep.
 */
int oracle_sweep_times(int n, int n_gates, int n_terms, const char *pauli, const double *coeffs,
                       double *sec_per_gate, double *sec_per_term) {
    if (n < 1 || n > ORACLE_MAX_QUBITS || n_gates < 1 || n_terms < 1 || !pauli || !coeffs ||
        !sec_per_gate || !sec_per_term)
        return ORACLE_EINVAL;
    const size_t dim = (size_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * dim);
    cplx *out = (cplx *)malloc(sizeof(cplx) * dim);
    if (!psi || !out) { free(psi); free(out); return ORACLE_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < (int64_t)dim; ++x) { psi[x] = 0.0; out[x] = 0.0; }
    psi[0] = 1.0;
#ifdef _OPENMP
    double t0 = omp_get_wtime();
#else
    double t0 = 0.0;
#endif
    for (int g = 0; g < n_gates; ++g) apply_ry(psi, n, g % n, 0.1 + 0.01 * g);
#ifdef _OPENMP
    double t1 = omp_get_wtime();
#else
    double t1 = 0.0;
#endif
    int rc = ORACLE_OK;
    for (int k = 0; k < n_terms && !rc; ++k)
        rc = apply_pauli_term(out, psi, n, pauli + (size_t)k * (size_t)n, coeffs[k]);
#ifdef _OPENMP
    double t2 = omp_get_wtime();
#else
    double t2 = 0.0;
#endif
    *sec_per_gate = (t1 - t0) / n_gates;
    *sec_per_term = (t2 - t1) / n_terms;
    free(psi);
    free(out);
    return rc;
}
