/*
 * rcg_oracle.c -- plain, slow FP64 CPU oracle of the regularized colour-gradient
 * lattice Boltzmann step for two immiscible components (Montessori et al.,
 * "Regularized lattice Boltzmann multicomponent models for low Capillary and
 * Reynolds microfluidics flows", arXiv:1711.02003).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or helper with the CUDA library; it is written straight from the paper's
 * equations in the paper's order and notation:
 *
 *   Eq. 1   f_i^k(x + c_i, t + 1) = f_i^k(x, t) + Omega_i^k          (stream + collide)
 *   Eq. 2   rho^k = sum_i f_i^k
 *   Eq. 3   rho u = sum_i sum_k f_i^k c_i
 *   Eq. 4   Omega = Omega^(3) [ Omega^(1) + Omega^(2) ]              (composition)
 *   Eq. 5   Omega^(1): relaxation towards f^eq
 *   Eq. 6   f_i^{k,eq} = rho^k [ phi_i^k + w_i (c.u/cs2 + (c.u)^2/(2 cs2^2) - u^2/(2 cs2)) ]
 *   Eq. 7   phi_i^k = alpha_k, (1-alpha_k)/5 (axis), (1-alpha_k)/20 (diagonal)   (D2Q9)
 *   Eq. 8   p^k = 3 rho^k (1 - alpha_k) / 5
 *   Eq. 9   Omega^(2): + (A/2)|F| [ w_i (F.c_i)^2/|F|^2 - B_i ]       (perturbation)
 *   Eq. 10  Omega^(3): recolouring with beta, cos(phi_i), sum_k f^{k,eq}(rho^k, 0, alpha_k)
 *   Eq. 11  regularization: post-collision rebuilt from rho, rho u and Pi only
 *
 * Readings taken where the paper is silent, ambiguous or garbled (each listed in
 * the design notes of the repository):
 *   R1  Eq. 4 is applied as a sequence: relax, then perturb, then recolour.
 *   R2  relaxation and perturbation act on the total f_i = sum_k f_i^k with one
 *       mixture relaxation time; only recolouring splits the components.
 *   R3  mixture viscosity: 1/nu = (1+psi)/(2 nu_R) + (1-psi)/(2 nu_B), nu_k = (tau_k - 1/2)/3.
 *   R4  a single A acts on the total f.
 *   R5  B_i (not printed): D2Q9 (-4/27, 2/27 axis, 5/108 diagonal);
 *       D3Q19 (-1/3, 1/18 face, 1/36 edge).
 *   R6  F is the isotropic gradient of psi = (rho_R - rho_B)/rho:
 *       F = 3 sum_{i>0} w_i psi(x + c_i) c_i.
 *   R7  |F| <= 1e-10: no perturbation and cos(phi_i) = 0; cos(phi_0) = 0 always.
 *   R8  Eq. 11 is read as f*_i = f_i^eq + (1 - 1/tau) * 4.5 w_i (c_ia c_ib - delta_ab/3) Pi^neq_ab,
 *       with Pi^neq = sum_i (f_i - f_i^eq) c_i c_i.
 *   R9  recolouring uses the moments of the post-streaming populations.
 *   R10 D3Q19 phi_i^k = alpha_k, (1-alpha_k)/12 (face), (1-alpha_k)/24 (edge).
 *   R11 boundaries (the paper gives none): halfway bounce-back at walls, ghost
 *       sites for ports filled before streaming from the inward neighbour x'
 *       (velocity inlet: equilibrium at rho(x') with the port's colour and
 *       velocity plus the non-equilibrium of x'; pressure outlet: equilibrium at
 *       the imposed density plus the non-equilibrium of x'; zero-gradient
 *       outlet: copy of x').  psi at a wall is psi_wall; at a ghost it is the
 *       psi of the ghost's own populations.
 *
 * Populations are stored [k][i][site], site = x + nx*(y + ny*z), k = 0 red, 1 blue.
 * Compile with -ffp-contract=off (no fused multiply-add) and without fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 19
#define ORC_MAXPORTS 8
#define ORC_EPS_F 1e-10

/* ------------------------------------------------------------------ lattice */

typedef struct {
    int d, q;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    int opp[ORC_MAXQ];
    double B[ORC_MAXQ];
} orc_lattice;

static void lattice_d2q9(orc_lattice* L)
{
    /* rest, 4 axis, 4 diagonal; 0-based numbering of the paper's i = 1..9 */
    static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    memset(L, 0, sizeof(*L));
    L->d = 2;
    L->q = 9;
    for (int i = 0; i < 9; ++i) {
        L->c[i][0] = c[i][0];
        L->c[i][1] = c[i][1];
        L->c[i][2] = 0;
    }
}

static void lattice_d3q19(orc_lattice* L)
{
    static const int c[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    memset(L, 0, sizeof(*L));
    L->d = 3;
    L->q = 19;
    for (int i = 0; i < 19; ++i)
        for (int a = 0; a < 3; ++a) L->c[i][a] = c[i][a];
}

/* weights, opposite directions and B_i from |c_i|^2 */
static void lattice_finish(orc_lattice* L)
{
    for (int i = 0; i < L->q; ++i) {
        int c2 = L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2];
        if (L->d == 2) {
            L->w[i] = c2 == 0 ? 4.0 / 9.0 : (c2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
            L->B[i] = c2 == 0 ? -4.0 / 27.0 : (c2 == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
        } else {
            L->w[i] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
            L->B[i] = c2 == 0 ? -1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
        for (int j = 0; j < L->q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
}

static int lattice_make(int lattice, orc_lattice* L)
{
    if (lattice == 0)
        lattice_d2q9(L);
    else if (lattice == 1)
        lattice_d3q19(L);
    else
        return -1;
    lattice_finish(L);
    return 0;
}

/* Eq. 7 (D2Q9) and reading R10 (D3Q19): phi_i^k as a function of alpha_k */
static double phi_of(const orc_lattice* L, double alpha, int i)
{
    int c2 = L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2];
    if (c2 == 0) return alpha;
    if (L->d == 2) return c2 == 1 ? (1.0 - alpha) / 5.0 : (1.0 - alpha) / 20.0;
    return c2 == 1 ? (1.0 - alpha) / 12.0 : (1.0 - alpha) / 24.0;
}

/* Eq. 6: equilibrium of one component */
static void feq_component(const orc_lattice* L, double alpha, double rho_k, const double u[3], double* out)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        out[i] = rho_k * (phi_of(L, alpha, i) + L->w[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    }
}

/* ------------------------------------------------------------------ params */

typedef struct {
    int lattice;        /* 0 D2Q9, 1 D3Q19 */
    int nx, ny, nz;
    int periodic[3];
    int collision;      /* 0 regularized (Eq. 11), 1 plain BGK (Eq. 5) */
    double tau_r, tau_b;
    double alpha_r, alpha_b;
    double A, beta;
    double rho0;
    double psi_wall;
} orc_params;

typedef struct {
    int kind;           /* 0 velocity inlet, 1 pressure outlet, 2 zero-gradient outlet */
    int normal_axis;    /* inward normal: axis 0..2 */
    int normal_sign;    /* +1 or -1 */
    int profile;        /* 0 parabolic, 1 flat */
    double u_max;
    double rho;         /* inlet density or outlet density */
    double psi;         /* inlet colour: +1 red, -1 blue */
} orc_port;

/* ----------------------------------------------------- per-site operators */

/* Omega^(1) on the total f (reading R2), regularized per Eq. 11 / R8 or plain BGK (Eq. 5).
 * f: total post-streaming populations; feq: total equilibrium.  out: post-relaxation. */
static void relax_total(const orc_lattice* L, int collision, double omega, const double* f,
                        const double* feq, double* out)
{
    if (collision == 1) {
        for (int i = 0; i < L->q; ++i) out[i] = feq[i] + (1.0 - omega) * (f[i] - feq[i]);
        return;
    }
    double Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < L->q; ++i) {
        double fneq = f[i] - feq[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi[a][b] += fneq * L->c[i][a] * L->c[i][b];
    }
    for (int i = 0; i < L->q; ++i) {
        double qpi = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double Q = L->c[i][a] * L->c[i][b] - (a == b ? 1.0 / 3.0 : 0.0);
                qpi += Q * Pi[a][b];
            }
        out[i] = feq[i] + (1.0 - omega) * 4.5 * L->w[i] * qpi;
    }
}

/* Omega^(2), Eq. 9 with reading R4/R5/R7: the increment added to every direction */
static void perturbation(const orc_lattice* L, double A, const double F[3], double* delta)
{
    double fn = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    for (int i = 0; i < L->q; ++i) {
        if (fn <= ORC_EPS_F) {
            delta[i] = 0.0;
            continue;
        }
        double Fc = F[0] * L->c[i][0] + F[1] * L->c[i][1] + F[2] * L->c[i][2];
        delta[i] = 0.5 * A * fn * (L->w[i] * Fc * Fc / (fn * fn) - L->B[i]);
    }
}

/* Omega^(3), Eq. 10 with reading R7: splits the total f into red and blue */
static void recolour(const orc_lattice* L, double beta, double alpha_r, double alpha_b, double rho_r,
                     double rho_b, const double F[3], const double* f, double* out_r, double* out_b)
{
    double rho = rho_r + rho_b;
    double fn = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    double zero[3] = {0.0, 0.0, 0.0};
    double er[ORC_MAXQ], eb[ORC_MAXQ];
    feq_component(L, alpha_r, rho_r, zero, er);
    feq_component(L, alpha_b, rho_b, zero, eb);
    for (int i = 0; i < L->q; ++i) {
        double cosphi = 0.0;
        if (i != 0 && fn > ORC_EPS_F) {
            double Fc = F[0] * L->c[i][0] + F[1] * L->c[i][1] + F[2] * L->c[i][2];
            double cn = sqrt((double)(L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] +
                                      L->c[i][2] * L->c[i][2]));
            cosphi = Fc / (fn * cn);
        }
        double seg = beta * rho_r * rho_b / (rho * rho) * cosphi * (er[i] + eb[i]);
        out_r[i] = rho_r / rho * f[i] + seg;
        out_b[i] = rho_b / rho * f[i] - seg;
    }
}

/* reading R3 */
static double mixture_omega(const orc_params* p, double psi)
{
    double nu_r = (p->tau_r - 0.5) / 3.0;
    double nu_b = (p->tau_b - 0.5) / 3.0;
    double inv_nu = (1.0 + psi) / (2.0 * nu_r) + (1.0 - psi) / (2.0 * nu_b);
    double tau = 3.0 / inv_nu + 0.5;
    return 1.0 / tau;
}

/* Full collision at one site: Eqs. 2-3 moments, then R1 order (relax, perturb, recolour). */
static void collide_site(const orc_params* p, const orc_lattice* L, const double* fr, const double* fb,
                         const double F[3], double* out_r, double* out_b)
{
    double rho_r = 0.0, rho_b = 0.0, j[3] = {0.0, 0.0, 0.0};
    double f[ORC_MAXQ];
    for (int i = 0; i < L->q; ++i) {
        rho_r += fr[i];
        rho_b += fb[i];
    }
    for (int i = 0; i < L->q; ++i) {
        f[i] = fr[i] + fb[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * L->c[i][a];
    }
    double rho = rho_r + rho_b;
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double psi = (rho_r - rho_b) / rho;
    double omega = mixture_omega(p, psi);

    double er[ORC_MAXQ], eb[ORC_MAXQ], feq[ORC_MAXQ] = {0.0}, fstar[ORC_MAXQ], delta[ORC_MAXQ];
    feq_component(L, p->alpha_r, rho_r, u, er);
    feq_component(L, p->alpha_b, rho_b, u, eb);
    for (int i = 0; i < L->q; ++i) feq[i] = er[i] + eb[i];
    relax_total(L, p->collision, omega, f, feq, fstar);
    perturbation(L, p->A, F, delta);
    for (int i = 0; i < L->q; ++i) fstar[i] += delta[i];
    recolour(L, p->beta, p->alpha_r, p->alpha_b, rho_r, rho_b, F, fstar, out_r, out_b);
}

/* ------------------------------------------------------------ public per-site entry points
 * (used by the closed-form pins in the test-suite)                                   */

int orc_lattice_tables(int lattice, int* c /* q*3 */, double* w, int* opp, double* B)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    for (int i = 0; i < L.q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
        B[i] = L.B[i];
    }
    return L.q;
}

int orc_phi(int lattice, double alpha, double* out)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    for (int i = 0; i < L.q; ++i) out[i] = phi_of(&L, alpha, i);
    return 0;
}

int orc_feq(int lattice, double alpha, double rho_k, const double* u, double* out)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    feq_component(&L, alpha, rho_k, u, out);
    return 0;
}

int orc_relax(int lattice, int collision, double omega, const double* f, const double* feq, double* out)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    relax_total(&L, collision, omega, f, feq, out);
    return 0;
}

int orc_perturbation(int lattice, double A, const double* F, double* delta)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    perturbation(&L, A, F, delta);
    return 0;
}

int orc_recolour(int lattice, double beta, double alpha_r, double alpha_b, double rho_r, double rho_b,
                 const double* F, const double* f, double* out_r, double* out_b)
{
    orc_lattice L;
    if (lattice_make(lattice, &L)) return -1;
    recolour(&L, beta, alpha_r, alpha_b, rho_r, rho_b, F, f, out_r, out_b);
    return 0;
}

double orc_mixture_omega(const orc_params* p, double psi) { return mixture_omega(p, psi); }

int orc_collide(const orc_params* p, const double* fr, const double* fb, const double* F, double* out_r,
                double* out_b)
{
    orc_lattice L;
    if (lattice_make(p->lattice, &L)) return -1;
    collide_site(p, &L, fr, fb, F, out_r, out_b);
    return 0;
}

/* ------------------------------------------------------------------ simulation */

typedef struct {
    orc_params p;
    orc_lattice L;
    long n;
    int dims[3];
    uint8_t* mask;     /* 0 fluid, 1 wall, 2+m ghost site of port m */
    orc_port ports[ORC_MAXPORTS];
    int nports;
    int lo[ORC_MAXPORTS][3], hi[ORC_MAXPORTS][3];
    double* A;         /* post-collision state [2][q][n] */
    double* Bf;        /* next state */
    double* fs;        /* post-streaming populations [2][q][n] */
    double* psi;       /* phase field of the current step, every site */
    long long step;
} orc_sim;

static long site_index(const orc_sim* s, int x, int y, int z)
{
    return (long)x + (long)s->dims[0] * ((long)y + (long)s->dims[1] * (long)z);
}

/* neighbour x + sgn*c_i; returns -1 when it leaves the box through a closed axis */
static long neighbour(const orc_sim* s, long site, int i, int sgn)
{
    int xyz[3];
    long r = site;
    xyz[0] = (int)(r % s->dims[0]);
    r /= s->dims[0];
    xyz[1] = (int)(r % s->dims[1]);
    xyz[2] = (int)(r / s->dims[1]);
    for (int a = 0; a < 3; ++a) {
        int v = xyz[a] + sgn * s->L.c[i][a];
        if (v < 0 || v >= s->dims[a]) {
            if (!s->p.periodic[a]) return -1;
            v = ((v % s->dims[a]) + s->dims[a]) % s->dims[a];
        }
        xyz[a] = v;
    }
    return site_index(s, xyz[0], xyz[1], xyz[2]);
}

static double* pop(double* base, const orc_sim* s, int k, int i) { return base + ((long)k * s->L.q + i) * s->n; }

void orc_sim_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->mask);
    free(s->A);
    free(s->Bf);
    free(s->fs);
    free(s->psi);
    free(s);
}

orc_sim* orc_sim_create(const orc_params* p, const uint8_t* mask, const orc_port* ports, int nports)
{
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->p = *p;
    if (lattice_make(p->lattice, &s->L)) {
        free(s);
        return NULL;
    }
    s->dims[0] = p->nx;
    s->dims[1] = p->ny;
    s->dims[2] = p->lattice == 0 ? 1 : p->nz;
    if (p->lattice == 0) s->p.periodic[2] = 1;
    s->n = (long)s->dims[0] * s->dims[1] * s->dims[2];
    if (nports < 0 || nports > ORC_MAXPORTS) {
        free(s);
        return NULL;
    }
    s->nports = nports;
    for (int m = 0; m < nports; ++m) s->ports[m] = ports[m];
    s->mask = (uint8_t*)malloc(s->n);
    s->A = (double*)calloc(2 * s->L.q * s->n, sizeof(double));
    s->Bf = (double*)calloc(2 * s->L.q * s->n, sizeof(double));
    s->fs = (double*)calloc(2 * s->L.q * s->n, sizeof(double));
    s->psi = (double*)calloc(s->n, sizeof(double));
    if (!s->mask || !s->A || !s->Bf || !s->fs || !s->psi) {
        orc_sim_destroy(s);
        return NULL;
    }
    memcpy(s->mask, mask, s->n);
    /* bounding box of each port's ghost sites: the extent of its velocity profile */
    for (int m = 0; m < nports; ++m)
        for (int a = 0; a < 3; ++a) {
            s->lo[m][a] = 1 << 30;
            s->hi[m][a] = -1;
        }
    for (long x = 0; x < s->n; ++x) {
        int code = s->mask[x];
        if (code < 2) continue;
        int m = code - 2;
        if (m >= nports) {
            orc_sim_destroy(s);
            return NULL;
        }
        int xyz[3] = {(int)(x % s->dims[0]), (int)((x / s->dims[0]) % s->dims[1]),
                      (int)(x / ((long)s->dims[0] * s->dims[1]))};
        for (int a = 0; a < 3; ++a) {
            if (xyz[a] < s->lo[m][a]) s->lo[m][a] = xyz[a];
            if (xyz[a] > s->hi[m][a]) s->hi[m][a] = xyz[a];
        }
    }
    return s;
}

/* velocity of a velocity-inlet ghost site: parabolic (or flat) over the port's
 * transverse extent, with the wall taken halfway between the last port site and
 * the wall site (s = coordinate - lo + 1/2). */
static void port_velocity(const orc_sim* s, int m, long g, double u[3])
{
    const orc_port* pt = &s->ports[m];
    int xyz[3] = {(int)(g % s->dims[0]), (int)((g / s->dims[0]) % s->dims[1]),
                  (int)(g / ((long)s->dims[0] * s->dims[1]))};
    double mag = pt->u_max;
    if (pt->profile == 0) {
        for (int a = 0; a < s->L.d; ++a) {
            if (a == pt->normal_axis) continue;
            double W = (double)(s->hi[m][a] - s->lo[m][a] + 1);
            double sc = (double)(xyz[a] - s->lo[m][a]) + 0.5;
            mag *= 4.0 * sc * (W - sc) / (W * W);
        }
    }
    u[0] = u[1] = u[2] = 0.0;
    u[pt->normal_axis] = mag * pt->normal_sign;
}

/* reading R11: fill the ghost sites of every port in the state A before streaming.
 * Velocity inlets and pressure outlets use non-equilibrium extrapolation from the
 * inward neighbour x' (Guo, Zheng and Shi 2002); zero-gradient outlets copy x'. */
static void fill_ports(orc_sim* s)
{
    const orc_lattice* L = &s->L;
    int q = L->q;
    for (long g = 0; g < s->n; ++g) {
        int code = s->mask[g];
        if (code < 2) continue;
        int m = code - 2;
        const orc_port* pt = &s->ports[m];
        /* inward neighbour x' = g + n */
        int xyz[3] = {(int)(g % s->dims[0]), (int)((g / s->dims[0]) % s->dims[1]),
                      (int)(g / ((long)s->dims[0] * s->dims[1]))};
        xyz[pt->normal_axis] += pt->normal_sign;
        long xp = site_index(s, xyz[0], xyz[1], xyz[2]);
        if (pt->kind == 2) {
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < q; ++i) pop(s->A, s, k, i)[g] = pop(s->A, s, k, i)[xp];
            continue;
        }
        /* moments of the inward neighbour's stored populations */
        double rr = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < q; ++i) {
            double a = pop(s->A, s, 0, i)[xp], b = pop(s->A, s, 1, i)[xp];
            rr += a;
            rb += b;
            for (int d = 0; d < 3; ++d) j[d] += (a + b) * L->c[i][d];
        }
        double rho = rr + rb;
        double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
        double er0[ORC_MAXQ], eb0[ORC_MAXQ], er1[ORC_MAXQ], eb1[ORC_MAXQ];
        feq_component(L, s->p.alpha_r, rr, u, er0);
        feq_component(L, s->p.alpha_b, rb, u, eb0);
        if (pt->kind == 0) {
            /* velocity inlet: equilibrium at the neighbour's density with the port's
             * colour and velocity, plus the neighbour's total non-equilibrium shared
             * out by the port's colour fractions */
            double ug[3];
            port_velocity(s, m, g, ug);
            double xr = (1.0 + pt->psi) / 2.0, xb = (1.0 - pt->psi) / 2.0;
            feq_component(L, s->p.alpha_r, xr * rho, ug, er1);
            feq_component(L, s->p.alpha_b, xb * rho, ug, eb1);
            for (int i = 0; i < q; ++i) {
                double fneq = pop(s->A, s, 0, i)[xp] + pop(s->A, s, 1, i)[xp] - (er0[i] + eb0[i]);
                pop(s->A, s, 0, i)[g] = er1[i] + xr * fneq;
                pop(s->A, s, 1, i)[g] = eb1[i] + xb * fneq;
            }
            continue;
        }
        /* pressure outlet: equilibrium at the imposed density with the neighbour's colour
         * fractions and velocity, plus the neighbour's per-component non-equilibrium */
        feq_component(L, s->p.alpha_r, pt->rho * rr / rho, u, er1);
        feq_component(L, s->p.alpha_b, pt->rho * rb / rho, u, eb1);
        for (int i = 0; i < q; ++i) {
            pop(s->A, s, 0, i)[g] = er1[i] + (pop(s->A, s, 0, i)[xp] - er0[i]);
            pop(s->A, s, 1, i)[g] = eb1[i] + (pop(s->A, s, 1, i)[xp] - eb0[i]);
        }
    }
}

/* Eq. 6 with u given: initial state f^{k,eq}(rho^k, u), treated as post-collision. */
int orc_sim_init_fields(orc_sim* s, const double* rho_r, const double* rho_b, const double* u /* d*n or NULL */)
{
    const orc_lattice* L = &s->L;
    for (long x = 0; x < s->n; ++x) {
        double uu[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < L->d; ++a) uu[a] = u[(long)a * s->n + x];
        double er[ORC_MAXQ], eb[ORC_MAXQ];
        int fluid = s->mask[x] == 0;
        feq_component(L, s->p.alpha_r, fluid ? rho_r[x] : 0.0, uu, er);
        feq_component(L, s->p.alpha_b, fluid ? rho_b[x] : 0.0, uu, eb);
        for (int i = 0; i < L->q; ++i) {
            pop(s->A, s, 0, i)[x] = er[i];
            pop(s->A, s, 1, i)[x] = eb[i];
        }
    }
    s->step = 0;
    return 0;
}

int orc_sim_set_populations(orc_sim* s, const double* f)
{
    memcpy(s->A, f, sizeof(double) * 2 * s->L.q * s->n);
    return 0;
}

int orc_sim_get_populations(const orc_sim* s, double* f)
{
    memcpy(f, s->A, sizeof(double) * 2 * s->L.q * s->n);
    return 0;
}

/* psi of a neighbour site for the colour gradient (readings R6, R11) */
static double psi_at(const orc_sim* s, long nb)
{
    if (nb < 0 || s->mask[nb] == 1) return s->p.psi_wall;
    return s->psi[nb];
}

static void step_once(orc_sim* s)
{
    const orc_lattice* L = &s->L;
    int q = L->q;
    long n = s->n;
    fill_ports(s);

    /* Eq. 1, streaming (pull) with halfway bounce-back at walls and closed box faces */
    long x;
#pragma omp parallel for schedule(static)
    for (x = 0; x < n; ++x) {
        if (s->mask[x] != 0) continue;
        for (int i = 0; i < q; ++i) {
            long src = neighbour(s, x, i, -1);
            int bounce = src < 0 || s->mask[src] == 1;
            for (int k = 0; k < 2; ++k)
                pop(s->fs, s, k, i)[x] = bounce ? pop(s->A, s, k, L->opp[i])[x] : pop(s->A, s, k, i)[src];
        }
    }

    /* Eqs. 2-3: densities and the phase field psi on fluid sites and port ghosts */
#pragma omp parallel for schedule(static)
    for (x = 0; x < n; ++x) {
        int code = s->mask[x];
        if (code == 1) continue;
        double *base = code == 0 ? s->fs : s->A;
        double rr = 0.0, rb = 0.0;
        for (int i = 0; i < q; ++i) {
            rr += pop(base, s, 0, i)[x];
            rb += pop(base, s, 1, i)[x];
        }
        s->psi[x] = (rr - rb) / (rr + rb);
    }

    /* colour gradient (R6) and collision (Eqs. 4-11) on fluid sites */
#pragma omp parallel for schedule(static)
    for (x = 0; x < n; ++x) {
        if (s->mask[x] != 0) continue;
        double F[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < q; ++i) {
            double ps = psi_at(s, neighbour(s, x, i, +1));
            for (int a = 0; a < 3; ++a) F[a] += L->w[i] * ps * L->c[i][a];
        }
        for (int a = 0; a < 3; ++a) F[a] *= 3.0;
        double fr[ORC_MAXQ], fb[ORC_MAXQ], outr[ORC_MAXQ], outb[ORC_MAXQ];
        for (int i = 0; i < q; ++i) {
            fr[i] = pop(s->fs, s, 0, i)[x];
            fb[i] = pop(s->fs, s, 1, i)[x];
        }
        collide_site(&s->p, L, fr, fb, F, outr, outb);
        for (int i = 0; i < q; ++i) {
            pop(s->Bf, s, 0, i)[x] = outr[i];
            pop(s->Bf, s, 1, i)[x] = outb[i];
        }
    }
    double* t = s->A;
    s->A = s->Bf;
    s->Bf = t;
    s->step += 1;
}

int orc_sim_step(orc_sim* s, long long nsteps)
{
    for (long long t = 0; t < nsteps; ++t) step_once(s);
    return 0;
}

long long orc_sim_step_count(const orc_sim* s) { return s->step; }

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Eqs. 2-3 on the stored state: rho_R, rho_B, u (d*n).  Non-fluid sites give zeros. */
int orc_sim_fields(const orc_sim* s, double* rho_r, double* rho_b, double* u)
{
    const orc_lattice* L = &s->L;
    for (long x = 0; x < s->n; ++x) {
        double rr = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
        if (s->mask[x] == 0) {
            for (int i = 0; i < L->q; ++i) {
                double a = pop(s->A, s, 0, i)[x], b = pop(s->A, s, 1, i)[x];
                rr += a;
                rb += b;
                for (int d = 0; d < 3; ++d) j[d] += (a + b) * L->c[i][d];
            }
        }
        rho_r[x] = rr;
        rho_b[x] = rb;
        double rho = rr + rb;
        for (int d = 0; d < L->d; ++d) u[(long)d * s->n + x] = rho > 0.0 ? j[d] / rho : 0.0;
    }
    return 0;
}

/* Observables on the stored state (fluid sites only).
 * out: [0] mass_R  [1] mass_B  [2..4] momentum  [5] p_in  [6] p_out  [7] dp
 *      [8] R_eff   [9] max|u|  [10] droplet amount sum (1+psi)/2  [11] n_in  [12] n_out
 * Pressure per Eq. 8 (D2Q9) or rho^k (1-alpha_k)/2 (D3Q19, reading R10).
 * r_in < 0 means R_eff/2, r_out < 0 means R_eff + 5 (interface width about 5 lattice units). */
int orc_sim_observables(const orc_sim* s, const double* centre, double r_in, double r_out, double* out)
{
    const orc_lattice* L = &s->L;
    int d = L->d;
    double mr = 0.0, mb = 0.0, mom[3] = {0.0, 0.0, 0.0}, amount = 0.0, umax = 0.0;
    double kp_r = d == 2 ? 3.0 * (1.0 - s->p.alpha_r) / 5.0 : (1.0 - s->p.alpha_r) / 2.0;
    double kp_b = d == 2 ? 3.0 * (1.0 - s->p.alpha_b) / 5.0 : (1.0 - s->p.alpha_b) / 2.0;
    for (long x = 0; x < s->n; ++x) {
        if (s->mask[x] != 0) continue;
        double rr = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < L->q; ++i) {
            double a = pop(s->A, s, 0, i)[x], b = pop(s->A, s, 1, i)[x];
            rr += a;
            rb += b;
            for (int k = 0; k < 3; ++k) j[k] += (a + b) * L->c[i][k];
        }
        double rho = rr + rb;
        mr += rr;
        mb += rb;
        for (int k = 0; k < 3; ++k) mom[k] += j[k];
        amount += (1.0 + (rr - rb) / rho) / 2.0;
        double u2 = (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / (rho * rho);
        double um = sqrt(u2);
        if (um > umax) umax = um;
    }
    double reff = d == 2 ? sqrt(amount / M_PI) : cbrt(3.0 * amount / (4.0 * M_PI));
    if (r_in < 0.0) r_in = reff / 2.0;
    if (r_out < 0.0) r_out = reff + 5.0;
    double pin = 0.0, pout = 0.0, nin = 0.0, nout = 0.0;
    for (long x = 0; x < s->n; ++x) {
        if (s->mask[x] != 0) continue;
        int xyz[3] = {(int)(x % s->dims[0]), (int)((x / s->dims[0]) % s->dims[1]),
                      (int)(x / ((long)s->dims[0] * s->dims[1]))};
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
            double dd = fabs((double)xyz[a] - centre[a]);
            if (s->p.periodic[a] && s->dims[a] - dd < dd) dd = s->dims[a] - dd;
            r2 += dd * dd;
        }
        double r = sqrt(r2);
        if (r >= r_in && r <= r_out) continue;
        double rr = 0.0, rb = 0.0;
        for (int i = 0; i < L->q; ++i) {
            rr += pop(s->A, s, 0, i)[x];
            rb += pop(s->A, s, 1, i)[x];
        }
        double pr = kp_r * rr + kp_b * rb;
        if (r < r_in) {
            pin += pr;
            nin += 1.0;
        } else {
            pout += pr;
            nout += 1.0;
        }
    }
    out[0] = mr;
    out[1] = mb;
    out[2] = mom[0];
    out[3] = mom[1];
    out[4] = mom[2];
    out[5] = nin > 0.0 ? pin / nin : 0.0;
    out[6] = nout > 0.0 ? pout / nout : 0.0;
    out[7] = out[5] - out[6];
    out[8] = reff;
    out[9] = umax;
    out[10] = amount;
    out[11] = nin;
    out[12] = nout;
    return 0;
}

/* Droplet labelling: connected components of {fluid and rho_R > rho_B} (psi > 0),
 * face-connected, periodic axes wrap.  Label = smallest linear index in the
 * component; -1 elsewhere.  Breadth-first search from each unlabelled site in
 * index order, so the first site reached is the smallest.  counts/volumes per
 * droplet in label order (volume = sum of (1+psi)/2).  Returns the number of
 * droplets (possibly > cap: only the first cap are written). */
int orc_sim_label(const orc_sim* s, int32_t* labels, int64_t* counts, double* volumes, int cap)
{
    const orc_lattice* L = &s->L;
    long n = s->n;
    char* drop = (char*)malloc(n);
    double* half = (double*)malloc(sizeof(double) * n);
    long* queue = (long*)malloc(sizeof(long) * n);
    if (!drop || !half || !queue) {
        free(drop);
        free(half);
        free(queue);
        return -1;
    }
    for (long x = 0; x < n; ++x) {
        labels[x] = -1;
        drop[x] = 0;
        half[x] = 0.0;
        if (s->mask[x] != 0) continue;
        double rr = 0.0, rb = 0.0;
        for (int i = 0; i < L->q; ++i) {
            rr += pop(s->A, s, 0, i)[x];
            rb += pop(s->A, s, 1, i)[x];
        }
        drop[x] = rr > rb;
        half[x] = (1.0 + (rr - rb) / (rr + rb)) / 2.0;
    }
    /* face neighbours are the directions with |c|^2 = 1 */
    int faces[6], nf = 0;
    for (int i = 0; i < L->q; ++i)
        if (abs(L->c[i][0]) + abs(L->c[i][1]) + abs(L->c[i][2]) == 1) faces[nf++] = i;
    int nd = 0;
    for (long x = 0; x < n; ++x) {
        if (!drop[x] || labels[x] >= 0) continue;
        long head = 0, tail = 0;
        queue[tail++] = x;
        labels[x] = (int32_t)x;
        int64_t cnt = 0;
        double vol = 0.0;
        while (head < tail) {
            long y = queue[head++];
            cnt += 1;
            for (int f = 0; f < nf; ++f) {
                long z = neighbour(s, y, faces[f], +1);
                if (z < 0 || !drop[z] || labels[z] >= 0) continue;
                labels[z] = (int32_t)x;
                queue[tail++] = z;
            }
        }
        /* volume summed in index order over the component's sites */
        for (long y = x; y < n; ++y)
            if (labels[y] == (int32_t)x) vol += half[y];
        if (nd < cap) {
            counts[nd] = cnt;
            volumes[nd] = vol;
        }
        nd += 1;
    }
    free(drop);
    free(half);
    free(queue);
    return nd;
}

/* Labelling of a bare boolean field (tests): same rule as orc_sim_label. */
int orc_label_field(int d, const int* dims, const int* periodic, const uint8_t* in, int32_t* labels)
{
    long n = (long)dims[0] * dims[1] * (d == 3 ? dims[2] : 1);
    long* queue = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
    if (!queue) return -1;
    int nd = 0;
    for (long x = 0; x < n; ++x) labels[x] = -1;
    for (long x = 0; x < n; ++x) {
        if (!in[x] || labels[x] >= 0) continue;
        long head = 0, tail = 0;
        queue[tail++] = x;
        labels[x] = (int32_t)x;
        while (head < tail) {
            long y = queue[head++];
            int xyz[3] = {(int)(y % dims[0]), (int)((y / dims[0]) % dims[1]),
                          d == 3 ? (int)(y / ((long)dims[0] * dims[1])) : 0};
            for (int a = 0; a < d; ++a)
                for (int sg = -1; sg <= 1; sg += 2) {
                    int v[3] = {xyz[0], xyz[1], xyz[2]};
                    v[a] += sg;
                    if (v[a] < 0 || v[a] >= dims[a]) {
                        if (!periodic[a]) continue;
                        v[a] = (v[a] + dims[a]) % dims[a];
                    }
                    long z = (long)v[0] + (long)dims[0] * ((long)v[1] + (long)dims[1] * v[2]);
                    if (!in[z] || labels[z] >= 0) continue;
                    labels[z] = (int32_t)x;
                    queue[tail++] = z;
                }
        }
        nd += 1;
    }
    free(queue);
    return nd;
}
