/*
 * acs_oracle.c -- plain FP64 CPU oracle for the RLB-MIE-FD time step of the
 * d-dimensional Allen-Cahn equation (Chen, Liu, Chai, Shi, arXiv:2312.07010).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes, each function citing the passage it follows:
 *   acs_oracle_cubic_root   Remark 1 (Eq. qtehta / Eq. root): the unique real root
 *                           of theta + (dt/2) f(theta) = xi, f(x) = x^3 - x.
 *   acs_oracle_step_fd      Eq. (IE-FD) / Eq. (IE-FD-vector-form): one step of the
 *                           finite-difference form, boundary per Eq. (Ddeltax).
 *   acs_oracle_step_lb      Eqs. (fieq-Fi), (fneq), (RLB), (pine): one step of the
 *                           regularized collide-and-stream form, summed over the
 *                           2d+1 populations, then the Remark 1 cubic.
 *   acs_oracle_energy       Theorem 3, Eq. (proof2-eq0): the discrete free energy.
 *   acs_oracle_maxnorm      Theorem 2 (the maximum norm over the unknowns).
 *   acs_oracle_adjoint_step transpose of the Jacobian of one step of Eq. (IE-FD),
 *                           plus that step's contribution to dL/d(eps^2).
 *
 * Grid convention (Eq. IE-FD-vector-form orders Phi with the last index fastest):
 * dims d in {1,2,3}; n[0..d-1] unknowns per axis; flat index
 * ((i0 * n1) + i1) * n2 + i2.  Outside an axis the neighbour ("ghost") value is
 *   periodic  : wrap around (the corner entries of the P-BC matrix D),
 *   Neumann   : the node itself (the -1 diagonal entries of the HN-BC matrix D),
 *   Dirichlet : zero (the HD-BC matrix D with the boundary values removed).
 *
 * Floating point: plain IEEE FP64.  Build with -ffp-contract=off so that x86-64
 * and aarch64 produce the same bits.  The per-point loops of the stepper carry an
 * OpenMP pragma; every point is independent, so the thread count changes timing
 * only, never a result.  Reductions are single-threaded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BC_PERIODIC 0
#define ORC_BC_NEUMANN 1
#define ORC_BC_DIRICHLET 2

typedef struct {
    int d;
    int64_t n[3];
    int64_t st[3];
    int64_t total;
} orc_grid;

static int orc_grid_init(orc_grid* g, int dims, const int64_t* n) {
    if (dims < 1 || dims > 3) return -1;
    g->d = dims;
    g->total = 1;
    for (int k = 0; k < 3; ++k) { g->n[k] = 1; g->st[k] = 0; }
    for (int k = 0; k < dims; ++k) {
        if (n[k] < 1) return -1;
        g->n[k] = n[k];
        g->total *= n[k];
    }
    int64_t s = 1;
    for (int k = dims - 1; k >= 0; --k) { g->st[k] = s; s *= g->n[k]; }
    return 0;
}

static void orc_coords(const orc_grid* g, int64_t idx, int64_t* c) {
    for (int k = g->d - 1; k >= 0; --k) { c[k] = idx % g->n[k]; idx /= g->n[k]; }
}

/* Value of the neighbour of node idx (coordinates c) one step along axis k in
 * direction dir (+1 or -1), with the ghost rule of the boundary condition. */
static double orc_nbr(const double* phi, const orc_grid* g, const int64_t* c, int64_t idx,
                      int k, int dir, int bc) {
    int64_t j = c[k] + dir;
    if (j >= 0 && j < g->n[k]) return phi[idx + dir * g->st[k]];
    if (bc == ORC_BC_PERIODIC) {
        int64_t jw = (j < 0) ? j + g->n[k] : j - g->n[k];
        return phi[idx + (jw - c[k]) * g->st[k]];
    }
    if (bc == ORC_BC_NEUMANN) return phi[idx];
    return 0.0;
}

/* Sum over the d axes of (phi_{+k} + phi_{-k} - 2 phi): Delta x^2 times row idx of
 * Lambda_{Delta x} Phi (Eq. IE-FD, Eq. Ddeltax). */
static double orc_link_sum(const double* phi, const orc_grid* g, const int64_t* c, int64_t idx,
                           int bc) {
    double s = 0.0;
    for (int k = 0; k < g->d; ++k)
        s += orc_nbr(phi, g, c, idx, k, +1, bc) + orc_nbr(phi, g, c, idx, k, -1, bc) - 2.0 * phi[idx];
    return s;
}

int acs_oracle_numthreads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void acs_oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* lambda = eps^2 dt / dx^2 (the lattice number omega1/s, Eq. IE-FD-vector-form). */
double acs_oracle_lambda(double eps, double dt, double h) { return eps * eps * dt / (h * h); }

/*
 * Remark 1: theta solves p(theta) = theta + (dt/2)(theta^3 - theta) - xi = 0.
 * With a = dt/2 < 1, p'(theta) = 1 - a + 3 a theta^2 > 0, so the root is unique
 * on the whole real line and lies in [-|xi|/(1-a), |xi|/(1-a)] (because
 * |a theta^3 + (1-a) theta| >= (1-a)|theta|).  Newton's method from xi/(1-a),
 * kept inside a shrinking bracket (bisection whenever a Newton step leaves it),
 * run until the iterate stops moving or the bracket is two adjacent doubles.
 */
double acs_oracle_cubic_root(double dt, double xi) {
    const double a = 0.5 * dt;
    const double b = 1.0 - a;
    double lo = -fabs(xi) / b, hi = fabs(xi) / b;
    double th = xi / b;
    for (int it = 0; it < 400; ++it) {
        double p = (a * th * th + b) * th - xi;
        if (p == 0.0) return th;
        if (p < 0.0) lo = th; else hi = th;
        const double mid = 0.5 * (lo + hi);
        if (!(lo < mid && mid < hi)) break;          /* lo and hi are adjacent doubles */
        double nt = th - p / (3.0 * a * th * th + b);
        if (!(nt > lo && nt < hi)) nt = mid;
        if (nt == th) break;
        th = nt;
    }
    /* Of the final iterate and the bracket ends, return the smallest residual. */
    double best = th, rb = fabs((a * th * th + b) * th - xi);
    double cand[2] = {lo, hi};
    for (int i = 0; i < 2; ++i) {
        double r = fabs((a * cand[i] * cand[i] + b) * cand[i] - xi);
        if (r < rb) { rb = r; best = cand[i]; }
    }
    return best;
}

void acs_oracle_cubic_root_array(double dt, const double* xi, double* out, int64_t count) {
    for (int64_t i = 0; i < count; ++i) out[i] = acs_oracle_cubic_root(dt, xi[i]);
}

/*
 * One step of Eq. (IE-FD):
 *   xi = phi + lambda * sum_k (phi_{+k} + phi_{-k} - 2 phi) - (dt/2) f(phi),
 *   phi_new = root of theta + (dt/2) f(theta) = xi              (Remark 1).
 * scheme 0 = RLB-MIE-FD (the paper's scheme).  scheme 1 = the fully explicit
 * FEX-FD scheme of Remark 2: phi_new = phi + lambda * sum - dt f(phi).
 */
int acs_oracle_step_fd(int dims, const int64_t* n, int bc, double lam, double dt,
                       const double* phi, double* out, int scheme) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0 || bc < 0 || bc > 2) return -1;
    const double a = 0.5 * dt;
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < g.total; ++idx) {
        int64_t c[3];
        orc_coords(&g, idx, c);
        const double p = phi[idx];
        const double lap = orc_link_sum(phi, &g, c, idx, bc);
        const double f = p * p * p - p;
        if (scheme == 1) {
            out[idx] = p + lam * lap - dt * f;
        } else {
            const double xi = p + lam * lap - a * f;
            out[idx] = acs_oracle_cubic_root(dt, xi);
        }
    }
    return 0;
}

/* steps applications of acs_oracle_step_fd; the result is left in phi. */
int acs_oracle_run_fd(int dims, const int64_t* n, int bc, double lam, double dt, int64_t steps,
                      double* phi, double* tmp, int scheme) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0) return -1;
    double* src = phi;
    double* dst = tmp;
    for (int64_t s = 0; s < steps; ++s) {
        int rc = acs_oracle_step_fd(dims, n, bc, lam, dt, src, dst, scheme);
        if (rc) return rc;
        double* t = src; src = dst; dst = t;
    }
    if (src != phi) memcpy(phi, src, (size_t)g.total * sizeof(double));
    return 0;
}

/*
 * One step of the regularized collide-and-stream form (Sec. II):
 *   equilibrium   f_k^eq = omega_k phi,  source F_k = -omega_k f(phi)     (Eq. fieq-Fi)
 *   c = dx/dt, c_s^2 = 2 omega1 c^2, s = omega1 / lambda,  s_A = (1-s)/c_s^2
 *   regularized non-equilibrium part  c_k . Pi^ne = -dt c_s^2 (c_k . grad phi) / s  (Eq. fneq)
 *   per-link gradient along the streaming link from y to y + c_k dt     (Eq. pine)
 *       c_k . grad phi (y) = (phi(y + c_k dt) - phi(y)) / dt
 *   post-collision at the source y:  g_k(y) = f_k^eq(y) + s_A omega_k c_k . Pi^ne(y)
 *   stream + source (Eq. RLB):  f_k(x) - dt/2 F_k(x, t+dt) = g_k(x - c_k dt) + dt/2 F_k(x, t)
 *   sum over k, sum_k f_k = phi_new, sum_k F_k = -f(phi):
 *       phi_new + dt/2 f(phi_new) = sum_k g_k(x - c_k dt) - dt/2 f(phi(x)) =: xi
 * Boundaries: the layer of ghost nodes around the box holds the boundary value
 * (wrap, mirror or zero) and its populations collide and stream like any other.
 * The populations are stored on the extended (n+2)^d lattice; entries that no
 * interior node reads are NaN, so using one by mistake poisons the result.
 */
int acs_oracle_step_lb(int dims, const int64_t* n, int bc, double eps, double dt, double h,
                       double omega1, const double* phi, double* out) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0 || bc < 0 || bc > 2) return -1;
    const int d = dims;
    const int q = 2 * d + 1;
    /* extended lattice */
    int64_t ne[3] = {1, 1, 1}, se[3] = {0, 0, 0};
    int64_t etot = 1;
    for (int k = 0; k < d; ++k) { ne[k] = g.n[k] + 2; etot *= ne[k]; }
    {
        int64_t s = 1;
        for (int k = d - 1; k >= 0; --k) { se[k] = s; s *= ne[k]; }
    }
    double* pe = (double*)malloc((size_t)etot * sizeof(double));
    double* gk = (double*)malloc((size_t)etot * (size_t)q * sizeof(double));
    if (!pe || !gk) { free(pe); free(gk); return -3; }
    const double nanv = nan("");
    /* fill the extended field: interior values, face ghosts by the boundary rule */
    for (int64_t e = 0; e < etot; ++e) {
        int64_t ce[3] = {0, 0, 0}, r = e;
        for (int k = d - 1; k >= 0; --k) { ce[k] = r % ne[k]; r /= ne[k]; }
        int outside = 0, axis = -1;
        for (int k = 0; k < d; ++k)
            if (ce[k] == 0 || ce[k] == ne[k] - 1) { ++outside; axis = k; }
        if (outside == 0) {
            int64_t idx = 0;
            for (int k = 0; k < d; ++k) idx += (ce[k] - 1) * g.st[k];
            pe[e] = phi[idx];
        } else if (outside == 1) {
            /* face ghost along `axis`: the boundary rule applied to the adjacent node */
            int64_t c[3] = {0, 0, 0};
            for (int k = 0; k < d; ++k) c[k] = ce[k] - 1;
            int dir = (ce[axis] == 0) ? -1 : +1;
            c[axis] -= dir; /* the interior node next to the ghost */
            int64_t idx = 0;
            for (int k = 0; k < d; ++k) idx += c[k] * g.st[k];
            pe[e] = orc_nbr(phi, &g, c, idx, axis, dir, bc);
        } else {
            pe[e] = nanv; /* edges and corners are never read by a face-neighbour stencil */
        }
    }
    const double c_lat = h / dt;
    const double cs2 = 2.0 * omega1 * c_lat * c_lat;
    const double lam = eps * eps * dt / (h * h);
    const double s = omega1 / lam;
    const double sA = (1.0 - s) / cs2;
    const double w0 = 1.0 - 2.0 * d * omega1;
    /* collide: every extended node, every population whose downstream node exists */
    for (int64_t e = 0; e < etot; ++e) {
        gk[(size_t)e * q + 0] = w0 * pe[e];
        int64_t ce[3] = {0, 0, 0}, r = e;
        for (int k = d - 1; k >= 0; --k) { ce[k] = r % ne[k]; r /= ne[k]; }
        for (int k = 0; k < d; ++k) {
            for (int sgn = 0; sgn < 2; ++sgn) {
                int dir = sgn ? -1 : +1;
                int pop = 1 + k + (sgn ? d : 0); /* c_{k} = +c e_k, c_{k+d} = -c e_k (Eq. ci) */
                int64_t jn = ce[k] + dir;
                double val = nanv;
                if (jn >= 0 && jn < ne[k]) {
                    double down = pe[e + dir * se[k]];
                    double cgrad = (down - pe[e]) / dt;          /* c_k . grad phi (y) */
                    double cPi = -dt * cs2 * cgrad / s;          /* c_k . Pi^ne (y) */
                    val = omega1 * pe[e] + sA * omega1 * cPi;    /* f_k^eq + s_A w_k c_k.Pi^ne */
                }
                gk[(size_t)e * q + pop] = val;
            }
        }
    }
    /* stream into the interior nodes, add the explicit source, solve the cubic */
    const double a = 0.5 * dt;
    for (int64_t idx = 0; idx < g.total; ++idx) {
        int64_t c[3];
        orc_coords(&g, idx, c);
        int64_t e = 0;
        for (int k = 0; k < d; ++k) e += (c[k] + 1) * se[k];
        double sum = gk[(size_t)e * q + 0];
        for (int k = 0; k < d; ++k) {
            sum += gk[(size_t)(e - se[k]) * q + 1 + k];       /* +c e_k arrives from x - e_k */
            sum += gk[(size_t)(e + se[k]) * q + 1 + k + d];   /* -c e_k arrives from x + e_k */
        }
        const double p = phi[idx];
        const double xi = sum - a * (p * p * p - p);
        out[idx] = acs_oracle_cubic_root(dt, xi);
    }
    free(pe);
    free(gk);
    return 0;
}

/* Neumaier's compensated summation (Neumaier 1974). */
typedef struct { double s, c; } orc_sum;
static void orc_add(orc_sum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x; else a->c += (x - t) + a->s;
    a->s = t;
}

/*
 * Theorem 3, Eq. (proof2-eq0):
 *   E = dx^d [ 1/4 sum_i (phi_i^2 - 1)^2 - lambda/(2 dt) Phi^T Lambda Phi ],
 *   Lambda = dx^2 Lambda_{dx}, so (Lambda Phi)_i = sum_k (phi_{+k} + phi_{-k} - 2 phi_i).
 * The sum runs over the unknowns only.
 */
double acs_oracle_energy(int dims, const int64_t* n, int bc, double lam, double dt, double h,
                         const double* phi) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0) return nan("");
    orc_sum bulk = {0, 0}, quad = {0, 0};
    for (int64_t idx = 0; idx < g.total; ++idx) {
        int64_t c[3];
        orc_coords(&g, idx, c);
        const double p = phi[idx];
        const double w = p * p - 1.0;
        orc_add(&bulk, 0.25 * w * w);
        orc_add(&quad, p * orc_link_sum(phi, &g, c, idx, bc));
    }
    const double hd = pow(h, (double)dims);
    return hd * ((bulk.s + bulk.c) - lam / (2.0 * dt) * (quad.s + quad.c));
}

/* Theorem 2: max_i |phi_i| over the unknowns (NaN if any entry is NaN). */
double acs_oracle_maxnorm(int dims, const int64_t* n, const double* phi) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0) return nan("");
    double m = 0.0;
    for (int64_t i = 0; i < g.total; ++i) {
        double v = fabs(phi[i]);
        if (v != v) return v;
        if (v > m) m = v;
    }
    return m;
}

/*
 * Transpose of the Jacobian of one step of Eq. (IE-FD).  Per node the step is
 *   xi_i = phi_i + lambda S_i(phi) - a f(phi_i),  S_i = sum_k (phi_{+k} + phi_{-k} - 2 phi_i),
 *   theta_i + a f(theta_i) = xi_i,  a = dt/2,
 * so d theta_i / d xi_i = 1 / (1 + a f'(theta_i)), f'(x) = 3x^2 - 1, and
 *   d xi_i / d phi_j = [i == j] (1 - a f'(phi_i)) + lambda dS_i/dphi_j.
 * Given adj_np1 = dL/dphi^{n+1}:  mu_i = adj_np1_i / (1 + a f'(phi^{n+1}_i)),
 *   adj_n_j = sum_i mu_i d xi_i / d phi_j
 *          = mu_j (1 - a f'(phi^n_j)) + lambda (S^T mu)_j,
 * where S^T is the same ghost-rule stencil (the matrices D of Eq. Ddeltax are
 * symmetric).  Since lambda = eps^2 dt / dx^2 with dt and dx fixed,
 *   d xi_i / d(eps^2) = (dt / dx^2) S_i(phi^n),
 * and the return value is sum_i mu_i (dt/dx^2) S_i(phi^n), this step's share of
 * dL/d(eps^2).  mu is caller scratch of numel doubles.
 */
double acs_oracle_adjoint_step(int dims, const int64_t* n, int bc, double lam, double dt, double h,
                               const double* phi_n, const double* phi_np1, const double* adj_np1,
                               double* adj_n, double* mu) {
    orc_grid g;
    if (orc_grid_init(&g, dims, n) != 0) return nan("");
    const double a = 0.5 * dt;
    for (int64_t i = 0; i < g.total; ++i) {
        const double th = phi_np1[i];
        mu[i] = adj_np1[i] / (1.0 + a * (3.0 * th * th - 1.0));
    }
    orc_sum ge = {0, 0};
    for (int64_t j = 0; j < g.total; ++j) {
        int64_t c[3];
        orc_coords(&g, j, c);
        const double p = phi_n[j];
        adj_n[j] = mu[j] * (1.0 - a * (3.0 * p * p - 1.0)) + lam * orc_link_sum(mu, &g, c, j, bc);
        orc_add(&ge, mu[j] * (dt / (h * h)) * orc_link_sum(phi_n, &g, c, j, bc));
    }
    return ge.s + ge.c;
}
