/* Plain FP64 spectral-element oracle in C with OpenMP: the multi-core CPU
 * restatement of what oracle/sem.py computes.
 *
 * TEST INFRASTRUCTURE ONLY (like the rest of oracle/): tests/ pin it against
 * the NumPy oracle and bench.py times it as the CPU baseline. It shares no
 * code with the CUDA library and includes none of its headers.
 *
 * What it computes (Section 4.1-4.2 of Araujo, Gross, Xavier-de-Souza 2021,
 * in the second-order form with the leapfrog, as the NumPy oracle states):
 *   - at every GLL point q = j (p+1) + i of element e, the Jacobian of the
 *     bilinear quad map, J = [dx/dxi dx/deta; dy/dxi dy/deta], its
 *     determinant and inverse (Eq. deriv_u with K^(e) = J^-1);
 *   - the per-point metric G_q = w_q |J_q| / rho_e J_q^-1 J_q^-T;
 *   - the dense element stiffness K_e[a][b] = sum_q B_q[:,a]^T G_q B_q[:,b]
 *     (B_q[d][a] the reference derivative of basis function a at point q,
 *     from the GLL derivative matrix), no sum factorisation;
 *   - the lumped mass M_nu = sum_{(e,q) -> nu} w_q |J_q| / (rho_e c_e^2)
 *     (Eq. Abar with the mass 1/K);
 *   - (K u)_nu = sum over the slots (e, q) of node nu, in ascending (e, q)
 *     order, of r_e[q] = sum_b K_e[q][b] u[conn[e][b]]: element residuals
 *     first (one thread per element), then one sum per node in a fixed order
 *     (one thread per node), so the result does not depend on the number of
 *     threads;
 *   - the leapfrog u^{n+1} = (2 u^n - u^{n-1}) + dt^2 (M^-1 (f(t_n) e_s - K u^n))
 *     with the source value f(t_n) passed in per step (Algorithm 3's point
 *     source at one node), and FP64 traces u^{n+1} at receiver nodes.
 * Build with -ffp-contract=off: every product and sum is rounded on its own,
 * as in NumPy.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t E, N;
    int np, P;
    int64_t* conn;     /* [E][P] global node of each slot (original numbering) */
    double* Ke;        /* [E][P][P] dense element stiffness */
    double* M;         /* [N] lumped mass */
    double* minv;      /* [N] 1 / M */
    int64_t* sptr;     /* [N+1] slots of each node, CSR */
    int64_t* slot;     /* [E*P] slot e*P+q, ascending within each node */
    double* r;         /* [E][P] element residuals (scratch) */
    double* ku;        /* [N] scratch */
    int threads;
} osem;

static void set_threads(const osem* s) {
#ifdef _OPENMP
    if (s->threads > 0) omp_set_num_threads(s->threads);
#else
    (void)s;
#endif
}

int osem_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void osem_destroy(osem* s) {
    if (!s) return;
    free(s->conn);
    free(s->Ke);
    free(s->M);
    free(s->minv);
    free(s->sptr);
    free(s->slot);
    free(s->r);
    free(s->ku);
    free(s);
}

/* coords[nv][2]; quads[E][4] counter-clockwise corners; conn[E][P] the
 * canonical numbering of the N global nodes; x, w the p+1 GLL nodes and
 * weights; D[i][k] = l_k'(x_i); vel, rho per element. Returns NULL on an
 * allocation failure or a non-positive Jacobian. */
osem* osem_create(const double* coords, const int64_t* quads, int64_t E, const int64_t* conn, int64_t N, int np,
                  const double* x, const double* w, const double* D, const double* vel, const double* rho,
                  int threads) {
    const int P = np * np;
    osem* s = (osem*)calloc(1, sizeof(osem));
    if (!s) return NULL;
    s->E = E;
    s->N = N;
    s->np = np;
    s->P = P;
    s->threads = threads;
    s->conn = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E * P));
    s->Ke = (double*)malloc(sizeof(double) * (size_t)(E * P * P));
    s->M = (double*)calloc((size_t)N, sizeof(double));
    s->minv = (double*)malloc(sizeof(double) * (size_t)N);
    s->sptr = (int64_t*)calloc((size_t)(N + 1), sizeof(int64_t));
    s->slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E * P));
    s->r = (double*)malloc(sizeof(double) * (size_t)(E * P));
    s->ku = (double*)malloc(sizeof(double) * (size_t)N);
    double* mloc = (double*)malloc(sizeof(double) * (size_t)(E * P));
    /* reference derivatives B[q][d][a] */
    double* B = (double*)calloc((size_t)(P * 2 * P), sizeof(double));
    if (!s->conn || !s->Ke || !s->M || !s->minv || !s->sptr || !s->slot || !s->r || !s->ku || !mloc || !B) {
        free(mloc);
        free(B);
        osem_destroy(s);
        return NULL;
    }
    memcpy(s->conn, conn, sizeof(int64_t) * (size_t)(E * P));
    for (int qj = 0; qj < np; ++qj)
        for (int qi = 0; qi < np; ++qi)
            for (int aj = 0; aj < np; ++aj)
                for (int ai = 0; ai < np; ++ai) {
                    const int q = qj * np + qi, a = aj * np + ai;
                    if (aj == qj) B[(q * 2 + 0) * P + a] = D[qi * np + ai]; /* d/dxi of l_ai(xi) l_aj(eta) */
                    if (ai == qi) B[(q * 2 + 1) * P + a] = D[qj * np + aj]; /* d/deta */
                }
    set_threads(s);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t e = 0; e < E; ++e) {
        double X[4], Y[4];
        for (int c = 0; c < 4; ++c) {
            X[c] = coords[quads[e * 4 + c] * 2];
            Y[c] = coords[quads[e * 4 + c] * 2 + 1];
        }
        double* K = s->Ke + (size_t)e * P * P;
        for (int k = 0; k < P * P; ++k) K[k] = 0.0;
        for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
                const int q = j * np + i;
                const double xi = x[i], eta = x[j];
                /* derivatives of the bilinear shape functions
                 * N0 = (1-xi)(1-eta)/4, N1 = (1+xi)(1-eta)/4,
                 * N2 = (1+xi)(1+eta)/4, N3 = (1-xi)(1+eta)/4 */
                const double dN_dxi[4] = {-0.25 * (1 - eta), 0.25 * (1 - eta), 0.25 * (1 + eta), -0.25 * (1 + eta)};
                const double dN_deta[4] = {-0.25 * (1 - xi), -0.25 * (1 + xi), 0.25 * (1 + xi), 0.25 * (1 - xi)};
                double J00 = 0, J01 = 0, J10 = 0, J11 = 0;
                for (int c = 0; c < 4; ++c) {
                    J00 += dN_dxi[c] * X[c];
                    J01 += dN_deta[c] * X[c];
                    J10 += dN_dxi[c] * Y[c];
                    J11 += dN_deta[c] * Y[c];
                }
                const double det = J00 * J11 - J01 * J10;
                if (!(det > 0.0)) bad = 1;
                /* J^-1 = adj(J) / det */
                const double I00 = J11 / det, I01 = -J01 / det, I10 = -J10 / det, I11 = J00 / det;
                /* J^-1 J^-T */
                const double m00 = I00 * I00 + I01 * I01;
                const double m01 = I00 * I10 + I01 * I11;
                const double m11 = I10 * I10 + I11 * I11;
                const double wq = w[i] * w[j];
                const double c = wq * det / rho[e];
                const double G[2][2] = {{c * m00, c * m01}, {c * m01, c * m11}};
                mloc[e * P + q] = wq * det / (rho[e] * (vel[e] * vel[e]));
                const double* Bq = B + (size_t)q * 2 * P;
                for (int a = 0; a < P; ++a)
                    for (int b = 0; b < P; ++b) {
                        double t = 0.0;
                        for (int d = 0; d < 2; ++d)
                            for (int k = 0; k < 2; ++k) t += Bq[d * P + a] * G[d][k] * Bq[k * P + b];
                        K[a * P + b] += t;
                    }
            }
    }
    free(B);
    if (bad) {
        free(mloc);
        osem_destroy(s);
        return NULL;
    }
    /* slots of each node, ascending (e, q): a counting sort over the slots */
    for (int64_t t = 0; t < E * P; ++t) s->sptr[conn[t] + 1] += 1;
    for (int64_t n = 0; n < N; ++n) s->sptr[n + 1] += s->sptr[n];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
        if (!fill) {
            free(mloc);
            osem_destroy(s);
            return NULL;
        }
        memcpy(fill, s->sptr, sizeof(int64_t) * (size_t)N);
        for (int64_t t = 0; t < E * P; ++t) s->slot[fill[conn[t]]++] = t;
        free(fill);
    }
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double acc = 0.0;
        for (int64_t k = s->sptr[n]; k < s->sptr[n + 1]; ++k) acc += mloc[s->slot[k]];
        s->M[n] = acc;
        s->minv[n] = 1.0 / acc;
    }
    free(mloc);
    return s;
}

/* Ku = K u (original numbering). */
static void apply_K(osem* s, const double* u, double* Ku) {
    const int P = s->P;
    const int64_t E = s->E, N = s->N;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        const double* K = s->Ke + (size_t)e * P * P;
        const int64_t* c = s->conn + e * P;
        double ue[81];
        for (int b = 0; b < P; ++b) ue[b] = u[c[b]];
        for (int a = 0; a < P; ++a) {
            double t = 0.0;
            for (int b = 0; b < P; ++b) t += K[a * P + b] * ue[b];
            s->r[e * P + a] = t;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double acc = 0.0;
        for (int64_t k = s->sptr[n]; k < s->sptr[n + 1]; ++k) acc += s->r[s->slot[k]];
        Ku[n] = acc;
    }
}

void osem_apply_K(osem* s, const double* u, double* Ku) {
    set_threads(s);
    apply_K(s, u, Ku);
}

void osem_mass(const osem* s, double* M) { memcpy(M, s->M, sizeof(double) * (size_t)s->N); }

/* nsteps leapfrog steps from (u, up) = (u^n, u^{n-1}), updated in place.
 * f[nsteps]: source values f(t_k) for the steps taken (ignored when
 * src_node < 0). traces[nrec][nsteps] (may be NULL when nrec = 0):
 * traces[r][k] = u^{k+1} at rec_nodes[r]. */
void osem_run(osem* s, int64_t nsteps, double dt, int64_t src_node, const double* f, const int64_t* rec_nodes,
              int32_t nrec, double* u, double* up, double* traces) {
    set_threads(s);
    const int64_t N = s->N;
    const double dt2 = dt * dt;
    for (int64_t k = 0; k < nsteps; ++k) {
        apply_K(s, u, s->ku);
        const double fk = src_node >= 0 ? f[k] : 0.0;
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            double rhs = -s->ku[n];
            if (n == src_node) rhs += fk;
            const double un = (2.0 * u[n] - up[n]) + dt2 * (s->minv[n] * rhs);
            up[n] = u[n];
            u[n] = un;
        }
        for (int32_t r = 0; r < nrec; ++r) traces[(int64_t)r * nsteps + k] = u[rec_nodes[r]];
    }
}
