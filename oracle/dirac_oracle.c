/*
 * FP64 CPU oracle for the multi-right-hand-side Dirac mat-vec of
 * S. Duerr, "Three Dirac operators on two architectures with one piece of
 * code and no hassle" (LATTICE 2018, arXiv:1808.05506).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is used by the tests, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py.  It shares no code with the CUDA path.
 *
 * What it computes, literally from the paper's definitions:
 *   staggered  D_S   (Sec. 3, the staggered definition and its eta phases) + m
 *   Wilson     D_W   (Sec. 4, Eq. def_wils with c_SW = 0, and the 2-point
 *                     derivative / 9-point Laplacian that follow it)
 *   Brillouin  D_B   (Sec. 5, Eqs. def_bril, def_der, def_lap with c_SW = 0,
 *                     coefficients rho_k, lambda_k printed after def_lap)
 *   W_dir            (Tab. tab:off-axis: the average over all k! hop orderings)
 * Every operator is written as the list of terms of one row y of the matrix
 * D(y, .): out(y) += coef * (S (x) C) psi(y + d), with S a spin matrix
 * (identity or gamma_mu) and C a colour matrix (a link, its adjoint, or W).
 * From that one list:
 *   apply          out(y)  = sum_terms coef S C psi(y+d)                 (gather)
 *   apply_dagger   out(x)  = sum_{d, y = x-d} conj(coef) S^+ C^+ psi(y)     (explicit adjoint,
 *                                                                         not via gamma5)
 *   force          dL/dV for L = Re <g, D psi>, PyTorch's complex convention
 *                  grad = dL/dRe V + i dL/dIm V, term by term.
 *
 * Readings where the paper is silent or misprinted (each a stated choice):
 *   - coordinates are 0-based, mu = 0..3 <-> x, y, z, t (array order of U);
 *     eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z).
 *   - periodic boundary conditions in all four directions.
 *   - V_{-mu}(x) = V_mu(x - mu)^dagger (the relation stated beside the
 *     2-point derivative of Sec. 4).
 *   - gamma matrices: Euclidean chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
 *     diag(1,1,-1,-1).
 *   - the sums over "mutually unequal" indices in def_der and def_lap run
 *     over unordered sets of distinct axes with both signs, so every offset
 *     appears once (this is what the 54-point and 81-point counts and the
 *     rho/lambda normalisations require).
 *   - def_der's rho_4 term couples through the 4-hop link W_{mu+nu+rho+sigma}
 *     (the printed W_{mu+nu+rho} is a misprint for a 4-hop offset).
 *   - Tab. tab:off-axis's 4-hop path ends with V_sigma(x+mu+nu+rho) (the
 *     printed argument x+mu+nu+sigma is a misprint: the path is ordered).
 *
 * Canonical layouts (C order, complex double):
 *   site  s = x + Nx (y + Ny (z + Nz t))
 *   V     [s][mu][a][b]
 *   psi   [s][v][spin][colour]      (Ns = 4 Wilson/Brillouin, Ns = 1 staggered)
 *   W81   [s][dir][a][b]            dir = sum_mu (d_mu + 1) 3^mu, d in {-1,0,1}^4
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>
#ifdef ORACLE_FP32
#include <tgmath.h>   /* conj, creal, cimag of float complex stay in float */
#endif

/* The oracle is FP64.  Compiled with -DORACLE_FP32 the same source gives a
 * single-precision instance (fields, links and arithmetic in float), used only
 * to time the CPU baseline in the paper's sp precision; the tests use FP64. */
#ifdef ORACLE_FP32
typedef float complex cplx;
typedef float real_t;
#else
typedef double complex cplx;
typedef double real_t;
#endif

enum { OP_STAGGERED = 0, OP_WILSON = 1, OP_BRILLOUIN = 2 };

typedef struct {
    int op, Nc, Ns, Nv;
    int L[4];
    long vol;
    double mass;             /* staggered m, Wilson m0, Brillouin m0 */
    const cplx* V;           /* links, canonical */
    const cplx* W;           /* Brillouin: W81 per site, or NULL (built per row) */
} ctx_t;

/* one term of row y: out(y) += coef * (S (x) C) psi(y + d) */
typedef struct {
    int d[4];
    cplx coef;
    int spin;                /* -1 identity, 0..3 gamma_mu */
    const cplx* C;           /* Nc x Nc row-major, NULL = identity */
    int dag;                 /* 1: use C^dagger */
    long link_site;          /* the gauge link C refers to (for the force), -1 if none */
    int link_mu;
} term_t;

#define MAX_TERMS 320
#define MAX_NC 8

/* ---- gamma matrices: Euclidean chiral basis ---------------------------- */
static cplx G[4][4][4];
static int g_init = 0;

static void init_gamma(void)
{
    if (g_init) return;
    /* Pauli matrices */
    cplx s[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[k][i][2 + j] = -I * s[k][i][j];
                G[k][2 + i][j] = I * s[k][i][j];
            }
    for (int i = 0; i < 2; ++i) {
        G[3][i][2 + i] = 1;
        G[3][2 + i][i] = 1;
    }
    g_init = 1;
}

void oracle_gamma(int mu, double* out /* 4x4 complex, interleaved */)
{
    init_gamma();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out[2 * (4 * i + j)] = creal(G[mu][i][j]);
            out[2 * (4 * i + j) + 1] = cimag(G[mu][i][j]);
        }
}

/* ---- lattice helpers ---------------------------------------------------- */
static void coords(const ctx_t* c, long s, int x[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(s % c->L[mu]);
        s /= c->L[mu];
    }
}

static long site_of(const ctx_t* c, const int x[4])
{
    long s = 0;
    for (int mu = 3; mu >= 0; --mu) {
        int v = ((x[mu] % c->L[mu]) + c->L[mu]) % c->L[mu];
        s = s * c->L[mu] + v;
    }
    return s;
}

static long shift(const ctx_t* c, long s, const int d[4])
{
    int x[4];
    coords(c, s, x);
    for (int mu = 0; mu < 4; ++mu) x[mu] += d[mu];
    return site_of(c, x);
}

static const cplx* link(const ctx_t* c, long s, int mu)
{
    return c->V + ((size_t)s * 4 + mu) * c->Nc * c->Nc;
}

static int dir_index(const int d[4])
{
    return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) + 27 * (d[3] + 1);
}

static void unit(int mu, int sign, int d[4])
{
    d[0] = d[1] = d[2] = d[3] = 0;
    d[mu] = sign;
}

static void push(term_t* T, int* n, const int d[4], cplx coef, int spin,
                 const cplx* C, int dag, long link_site, int link_mu)
{
    term_t* t = &T[(*n)++];
    memcpy(t->d, d, sizeof(t->d));
    t->coef = coef;
    t->spin = spin;
    t->C = C;
    t->dag = dag;
    t->link_site = link_site;
    t->link_mu = link_mu;
}

/* ---- small colour algebra ----------------------------------------------- */
static void mat_mul(int Nc, const cplx* A, int adag, const cplx* B, int bdag, cplx* out)
{
    for (int a = 0; a < Nc; ++a)
        for (int b = 0; b < Nc; ++b) {
            cplx acc = 0;
            for (int k = 0; k < Nc; ++k) {
                cplx x = adag ? conj(A[k * Nc + a]) : A[a * Nc + k];
                cplx y = bdag ? conj(B[b * Nc + k]) : B[k * Nc + b];
                acc += x * y;
            }
            out[a * Nc + b] = acc;
        }
}

/* ---- Tab. tab:off-axis: W_dir(y) = (1/k!) sum over the k! hop orderings --- */
/* One signed unit hop h = (axis, sign): V_h(z) = V_axis(z) for sign +1 and
 * V_{-axis}(z) = V_axis(z - axis)^dagger for sign -1; the hop moves z -> z+h. */
static void hop_link(const ctx_t* c, long z, int axis, int sign, cplx* out, long* znext)
{
    int Nc = c->Nc;
    int d[4];
    unit(axis, sign, d);
    if (sign > 0) {
        memcpy(out, link(c, z, axis), sizeof(cplx) * Nc * Nc);
    } else {
        const cplx* U = link(c, shift(c, z, d), axis);
        for (int a = 0; a < Nc; ++a)
            for (int b = 0; b < Nc; ++b) out[a * Nc + b] = conj(U[b * Nc + a]);
    }
    *znext = shift(c, z, d);
}

static void W_dir(const ctx_t* c, long y, const int d[4], cplx* W)
{
    int Nc = c->Nc;
    int axis[4], sign[4], k = 0;
    for (int mu = 0; mu < 4; ++mu)
        if (d[mu] != 0) {
            axis[k] = mu;
            sign[k] = d[mu];
            ++k;
        }
    memset(W, 0, sizeof(cplx) * Nc * Nc);
    if (k == 0) {
        for (int a = 0; a < Nc; ++a) W[a * Nc + a] = 1;
        return;
    }
    /* all orderings = all k-tuples of distinct hop indices */
    int npaths = 0;
    int ord[4];
    int total = 1;
    for (int i = 0; i < k; ++i) total *= k;
    for (int code = 0; code < total; ++code) {
        int cc = code, used = 0, ok = 1;
        for (int i = 0; i < k; ++i) {
            ord[i] = cc % k;
            cc /= k;
            if (used & (1 << ord[i])) ok = 0;
            used |= 1 << ord[i];
        }
        if (!ok) continue;
        cplx P[MAX_NC * MAX_NC], H[MAX_NC * MAX_NC], tmp[MAX_NC * MAX_NC];
        long z = y;
        for (int i = 0; i < k; ++i) {
            long zn;
            hop_link(c, z, axis[ord[i]], sign[ord[i]], H, &zn);
            if (i == 0) {
                memcpy(P, H, sizeof(cplx) * Nc * Nc);
            } else {
                mat_mul(Nc, P, 0, H, 0, tmp);
                memcpy(P, tmp, sizeof(cplx) * Nc * Nc);
            }
            z = zn;
        }
        for (int e = 0; e < Nc * Nc; ++e) W[e] += P[e];
        ++npaths;
    }
    for (int e = 0; e < Nc * Nc; ++e) W[e] /= (double)npaths;
}

/* all 81 directions at site y (dir 40 = the trivial one, identity) */
static void W81_site(const ctx_t* c, long y, cplx* W81)
{
    int Nc = c->Nc;
    for (int dir = 0; dir < 81; ++dir) {
        int d[4] = {dir % 3 - 1, (dir / 3) % 3 - 1, (dir / 9) % 3 - 1, (dir / 27) % 3 - 1};
        W_dir(c, y, d, W81 + (size_t)dir * Nc * Nc);
    }
}

/* ---- the rows of the three operators ------------------------------------ */

/* Sec. 3: D_S(y,.) = sum_mu eta_mu(y) 1/2 [V_mu(y) delta_{y+mu} - V_mu(y-mu)^+ delta_{y-mu}],
 * plus the mass term m delta_{y,y}. */
static int rows_staggered(const ctx_t* c, long y, term_t* T)
{
    int n = 0, x[4], d[4];
    coords(c, y, x);
    for (int mu = 0; mu < 4; ++mu) {
        int e = 0;
        for (int nu = 0; nu < mu; ++nu) e += x[nu];
        double eta = (e % 2) ? -1.0 : 1.0;
        unit(mu, +1, d);
        push(T, &n, d, 0.5 * eta, -1, link(c, y, mu), 0, y, mu);
        unit(mu, -1, d);
        long ym = shift(c, y, d);
        push(T, &n, d, -0.5 * eta, -1, link(c, ym, mu), 1, ym, mu);
    }
    int z[4] = {0, 0, 0, 0};
    push(T, &n, z, c->mass, -1, NULL, 0, -1, -1);
    return n;
}

/* Sec. 4, def_wils at c_SW = 0 (lattice spacing a = 1):
 *   sum_mu gamma_mu grad_mu^std  -  1/2 lap^std  +  m0,
 *   grad_mu^std(y,.) = 1/2 [V_mu(y) delta_{y+mu} - V_{-mu}(y) delta_{y-mu}],
 *   lap^std(y,.)     = -8 delta_{y,y} + sum over the 8 signed mu of V_mu(y) delta_{y+mu}. */
static int rows_wilson(const ctx_t* c, long y, term_t* T)
{
    int n = 0, d[4], z[4] = {0, 0, 0, 0};
    /* sum_mu gamma_mu grad_mu */
    for (int mu = 0; mu < 4; ++mu) {
        unit(mu, +1, d);
        push(T, &n, d, 0.5, mu, link(c, y, mu), 0, y, mu);
        unit(mu, -1, d);
        long ym = shift(c, y, d);
        push(T, &n, d, -0.5, mu, link(c, ym, mu), 1, ym, mu);
    }
    /* -1/2 lap */
    push(T, &n, z, -0.5 * -8.0, -1, NULL, 0, -1, -1);
    for (int mu = 0; mu < 4; ++mu) {
        unit(mu, +1, d);
        push(T, &n, d, -0.5, -1, link(c, y, mu), 0, y, mu);
        unit(mu, -1, d);
        long ym = shift(c, y, d);
        push(T, &n, d, -0.5, -1, link(c, ym, mu), 1, ym, mu);
    }
    /* m0 */
    push(T, &n, z, c->mass, -1, NULL, 0, -1, -1);
    return n;
}

static const double RHO[5] = {0.0, 64.0 / 432.0, 16.0 / 432.0, 4.0 / 432.0, 1.0 / 432.0};
static const double LAMBDA[5] = {-240.0 / 64.0, 8.0 / 64.0, 4.0 / 64.0, 2.0 / 64.0, 1.0 / 64.0};

static const cplx* Wat(const ctx_t* c, const cplx* W81, const int d[4])
{
    return W81 + (size_t)dir_index(d) * c->Nc * c->Nc;
}

/* Sec. 5, def_bril at c_SW = 0:  sum_mu gamma_mu grad_mu^iso - 1/2 lap^bri + m0.
 * grad_mu^iso (def_der): for each of the two brackets (+mu, then the
 * "-(mu -> -mu)" bracket entering with a minus sign): rho_1 W_{+-mu}, then
 * rho_2 over the 6 signed nu != mu, rho_3 over the unordered pairs of the
 * other axes with both signs, rho_4 over the remaining three axes with all
 * signs.  lap^bri (def_lap): lambda_0 delta + lambda_k over every k-hop
 * offset with pairwise unequal axes (each offset once). */
static int rows_brillouin(const ctx_t* c, long y, const cplx* W81, term_t* T)
{
    int n = 0, z[4] = {0, 0, 0, 0};
    for (int mu = 0; mu < 4; ++mu) {
        int oth[3], no = 0;
        for (int a = 0; a < 4; ++a)
            if (a != mu) oth[no++] = a;
        for (int smu = +1; smu >= -1; smu -= 2) {
            double br = (double)smu; /* +[...] for +mu, -[...] for the mirrored bracket */
            int d[4];
            /* rho_1 */
            unit(mu, smu, d);
            push(T, &n, d, br * RHO[1], mu, Wat(c, W81, d), 0, -1, -1);
            /* rho_2: nu over the other axes, both signs */
            for (int i = 0; i < 3; ++i)
                for (int sn = -1; sn <= 1; sn += 2) {
                    unit(mu, smu, d);
                    d[oth[i]] = sn;
                    push(T, &n, d, br * RHO[2], mu, Wat(c, W81, d), 0, -1, -1);
                }
            /* rho_3: unordered pairs {nu, rho} of the other axes, all signs */
            for (int i = 0; i < 3; ++i)
                for (int j = i + 1; j < 3; ++j)
                    for (int sn = -1; sn <= 1; sn += 2)
                        for (int sr = -1; sr <= 1; sr += 2) {
                            unit(mu, smu, d);
                            d[oth[i]] = sn;
                            d[oth[j]] = sr;
                            push(T, &n, d, br * RHO[3], mu, Wat(c, W81, d), 0, -1, -1);
                        }
            /* rho_4: nu, rho, sigma = the three other axes, all signs */
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2)
                    for (int sc = -1; sc <= 1; sc += 2) {
                        unit(mu, smu, d);
                        d[oth[0]] = sa;
                        d[oth[1]] = sb;
                        d[oth[2]] = sc;
                        push(T, &n, d, br * RHO[4], mu, Wat(c, W81, d), 0, -1, -1);
                    }
        }
    }
    /* -1/2 lap^bri */
    push(T, &n, z, -0.5 * LAMBDA[0], -1, NULL, 0, -1, -1);
    for (int dir = 0; dir < 81; ++dir) {
        int d[4] = {dir % 3 - 1, (dir / 3) % 3 - 1, (dir / 9) % 3 - 1, (dir / 27) % 3 - 1};
        int k = abs(d[0]) + abs(d[1]) + abs(d[2]) + abs(d[3]);
        if (k == 0) continue;
        push(T, &n, d, -0.5 * LAMBDA[k], -1, Wat(c, W81, d), 0, -1, -1);
    }
    /* m0 */
    push(T, &n, z, c->mass, -1, NULL, 0, -1, -1);
    return n;
}

/* rows of D at y; W81buf is per-thread scratch for Brillouin when c->W == NULL */
static int rows(const ctx_t* c, long y, term_t* T, cplx* W81buf)
{
    switch (c->op) {
    case OP_STAGGERED: return rows_staggered(c, y, T);
    case OP_WILSON: return rows_wilson(c, y, T);
    default: {
        const cplx* W81;
        if (c->W) {
            W81 = c->W + (size_t)y * 81 * c->Nc * c->Nc;
        } else {
            W81_site(c, y, W81buf);
            W81 = W81buf;
        }
        return rows_brillouin(c, y, W81, T);
    }
    }
}

/* out_site[v][s][a] += coef * sum_{s',b} S[s][s'] C[a][b] in_site[v][s'][b]  (or daggers) */
static void apply_term(const ctx_t* c, const term_t* t, int dagger,
                       const cplx* in_site, cplx* out_site)
{
    int Nc = c->Nc, Ns = c->Ns, Nv = c->Nv;
    cplx coef = dagger ? conj(t->coef) : t->coef;
    for (int v = 0; v < Nv; ++v)
        for (int s = 0; s < Ns; ++s)
            for (int a = 0; a < Nc; ++a) {
                cplx acc = 0;
                for (int sp = 0; sp < Ns; ++sp) {
                    cplx Sv;
                    if (t->spin < 0) Sv = (s == sp) ? 1.0 : 0.0;
                    else Sv = dagger ? conj(G[t->spin][sp][s]) : G[t->spin][s][sp];
                    if (Sv == 0) continue;
                    for (int b = 0; b < Nc; ++b) {
                        cplx Cv;
                        if (!t->C) Cv = (a == b) ? 1.0 : 0.0;
                        else {
                            int use_dag = t->dag ^ dagger;
                            Cv = use_dag ? conj(t->C[b * Nc + a]) : t->C[a * Nc + b];
                        }
                        acc += Sv * Cv * in_site[((size_t)v * Ns + sp) * Nc + b];
                    }
                }
                out_site[((size_t)v * Ns + s) * Nc + a] += coef * acc;
            }
}

static void set_ctx(ctx_t* c, int op, int Nc, const int* L, int Nv, double mass,
                    const real_t* V, const real_t* W)
{
    init_gamma();
    c->op = op;
    c->Nc = Nc;
    c->Ns = (op == OP_STAGGERED) ? 1 : 4;
    c->Nv = Nv;
    for (int mu = 0; mu < 4; ++mu) c->L[mu] = L[mu];
    c->vol = (long)L[0] * L[1] * L[2] * L[3];
    c->mass = mass;
    c->V = (const cplx*)V;
    c->W = (const cplx*)W;
}

/* ---- public entry points ------------------------------------------------ */

/* OpenMP threads of the parallel loops below (n < 1: one per processor);
 * returns the number the next parallel region will use. */
int oracle_set_threads(int n)
{
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
    return omp_get_max_threads();
}

/* out = D psi (dagger = 0) or D^dagger psi (dagger = 1), at the listed output
 * sites (sites == NULL: all sites, out in canonical order); out is
 * [nsite][Nv][Ns][Nc].  W81 may be NULL for Brillouin (built per row). */
int oracle_apply(int op, int Nc, const int* L, int Nv, double mass, const real_t* V,
                 const real_t* W81, const real_t* psi, real_t* out,
                 const long* sites, long nsites, int dagger)
{
    if (Nc < 1 || Nc > MAX_NC) return 1;
    ctx_t c;
    set_ctx(&c, op, Nc, L, Nv, mass, V, W81);
    if (!sites) nsites = c.vol;
    const cplx* in = (const cplx*)psi;
    cplx* o = (cplx*)out;
    size_t blk = (size_t)Nv * c.Ns * Nc;
    memset(o, 0, sizeof(cplx) * blk * nsites);
#pragma omp parallel
    {
        term_t* T = malloc(sizeof(term_t) * MAX_TERMS);
        cplx* W81buf = (op == OP_BRILLOUIN && !W81) ? malloc(sizeof(cplx) * 81 * Nc * Nc) : NULL;
        cplx* W81buf2 = (op == OP_BRILLOUIN && !W81) ? malloc(sizeof(cplx) * 81 * Nc * Nc) : NULL;
#pragma omp for schedule(dynamic, 16)
        for (long i = 0; i < nsites; ++i) {
            long x = sites ? sites[i] : i;
            cplx* ox = o + blk * i;
            if (!dagger) {
                int nt = rows(&c, x, T, W81buf);
                for (int k = 0; k < nt; ++k)
                    apply_term(&c, &T[k], 0, in + blk * shift(&c, x, T[k].d), ox);
            } else {
                /* (D^+ psi)(x) = sum_y D(y,x)^+ psi(y): visit every row y = x - d
                 * that can reach x and keep its terms with offset d. */
                for (int dir = 0; dir < 81; ++dir) {
                    int d[4] = {dir % 3 - 1, (dir / 3) % 3 - 1, (dir / 9) % 3 - 1, (dir / 27) % 3 - 1};
                    int k = abs(d[0]) + abs(d[1]) + abs(d[2]) + abs(d[3]);
                    if (op != OP_BRILLOUIN && k > 1) continue;
                    int md[4] = {-d[0], -d[1], -d[2], -d[3]};
                    long y = shift(&c, x, md);
                    int nt = rows(&c, y, T, W81buf2);
                    for (int t = 0; t < nt; ++t) {
                        if (T[t].d[0] != d[0] || T[t].d[1] != d[1] || T[t].d[2] != d[2] ||
                            T[t].d[3] != d[3])
                            continue;
                        apply_term(&c, &T[t], 1, in + blk * y, ox);
                    }
                }
            }
        }
        free(T);
        free(W81buf);
        free(W81buf2);
    }
    return 0;
}

/* W_dir(y) for all 81 dir at the listed sites (sites == NULL: all), out [nsite][81][Nc][Nc] */
int oracle_brillouin_W(int Nc, const int* L, const real_t* V, const long* sites, long nsites,
                       real_t* out)
{
    if (Nc < 1 || Nc > MAX_NC) return 1;
    ctx_t c;
    set_ctx(&c, OP_BRILLOUIN, Nc, L, 1, 0.0, V, NULL);
    if (!sites) nsites = c.vol;
    cplx* o = (cplx*)out;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < nsites; ++i) W81_site(&c, sites ? sites[i] : i, o + (size_t)i * 81 * Nc * Nc);
    return 0;
}

/* M[b][a] = coef sum_{v,s,s'} psi_v(y+d)[s'][b] S[s][s'] conj(g_v(y)[s][a]) of one term */
static void term_M(const ctx_t* c, const term_t* t, const cplx* py, const cplx* gy, cplx* M)
{
    int Nc = c->Nc, Nv = c->Nv;
    for (int b = 0; b < Nc; ++b)
        for (int a = 0; a < Nc; ++a) {
            cplx acc = 0;
            for (int v = 0; v < Nv; ++v)
                for (int s = 0; s < c->Ns; ++s)
                    for (int sp = 0; sp < c->Ns; ++sp) {
                        cplx Sv = (t->spin < 0) ? (s == sp ? 1.0 : 0.0) : G[t->spin][s][sp];
                        if (Sv == 0) continue;
                        acc += py[((size_t)v * c->Ns + sp) * Nc + b] * Sv * conj(gy[((size_t)v * c->Ns + s) * Nc + a]);
                    }
            M[b * Nc + a] = t->coef * acc;
        }
}

/* Brillouin: the terms couple through W_dir(y) = (1/k!) sum over the k! hop
 * orderings of the path products H_1 ... H_k (Tab. tab:off-axis), with
 * H = V_mu(z) for a +mu hop and V_mu(z - mu)^+ for a -mu hop.  The gradient
 * with respect to W_dir(y) is the sum of M^+ over the terms through W_dir(y);
 * for one ordering, Re tr(G^+ P1 H P2) gives P1^+ G P2^+ for H and, for a
 * -mu hop, its adjoint P2 G^+ P1 for V_mu(z - mu); each weighted 1/k!. */
static void brillouin_force(const ctx_t* c, const cplx* P, const cplx* Gv, cplx* Fo)
{
    int Nc = c->Nc;
    size_t n2 = (size_t)Nc * Nc, blk = (size_t)c->Nv * c->Ns * Nc;
    term_t T[MAX_TERMS];
    cplx* W81 = malloc(sizeof(cplx) * 81 * n2);
    cplx* G81 = malloc(sizeof(cplx) * 81 * n2);
    cplx M[MAX_NC * MAX_NC];
    for (long y = 0; y < c->vol; ++y) {
        W81_site(c, y, W81);
        int nt = rows_brillouin(c, y, W81, T);
        memset(G81, 0, sizeof(cplx) * 81 * n2);
        for (int t = 0; t < nt; ++t) {
            if (!T[t].C) continue;
            term_M(c, &T[t], P + blk * shift(c, y, T[t].d), Gv + blk * y, M);
            cplx* Gd = G81 + (size_t)dir_index(T[t].d) * n2;
            for (int a = 0; a < Nc; ++a)
                for (int b = 0; b < Nc; ++b) Gd[a * Nc + b] += conj(M[b * Nc + a]);
        }
        for (int dir = 0; dir < 81; ++dir) {
            int d[4] = {dir % 3 - 1, (dir / 3) % 3 - 1, (dir / 9) % 3 - 1, (dir / 27) % 3 - 1};
            int axis[4], sign[4], k = 0;
            for (int mu = 0; mu < 4; ++mu)
                if (d[mu] != 0) {
                    axis[k] = mu;
                    sign[k] = d[mu];
                    ++k;
                }
            if (k == 0) continue;
            const cplx* Gd = G81 + (size_t)dir * n2;
            double fact = 1;
            for (int i = 2; i <= k; ++i) fact *= i;
            int total = 1;
            for (int i = 0; i < k; ++i) total *= k;
            for (int code = 0; code < total; ++code) {
                int cc = code, used = 0, ok = 1, ord[4];
                for (int i = 0; i < k; ++i) {
                    ord[i] = cc % k;
                    cc /= k;
                    if (used & (1 << ord[i])) ok = 0;
                    used |= 1 << ord[i];
                }
                if (!ok) continue;
                cplx H[4][MAX_NC * MAX_NC];
                long z[5];
                z[0] = y;
                for (int i = 0; i < k; ++i) hop_link(c, z[i], axis[ord[i]], sign[ord[i]], H[i], &z[i + 1]);
                for (int i = 0; i < k; ++i) {
                    cplx P1[MAX_NC * MAX_NC], P2[MAX_NC * MAX_NC], tmp[MAX_NC * MAX_NC], X[MAX_NC * MAX_NC];
                    for (int e = 0; e < Nc * Nc; ++e) P1[e] = P2[e] = 0;
                    for (int a = 0; a < Nc; ++a) P1[a * Nc + a] = P2[a * Nc + a] = 1;
                    for (int j = 0; j < i; ++j) {
                        mat_mul(Nc, P1, 0, H[j], 0, tmp);
                        memcpy(P1, tmp, sizeof(cplx) * n2);
                    }
                    for (int j = i + 1; j < k; ++j) {
                        mat_mul(Nc, P2, 0, H[j], 0, tmp);
                        memcpy(P2, tmp, sizeof(cplx) * n2);
                    }
                    const int mu = axis[ord[i]];
                    if (sign[ord[i]] > 0) {
                        mat_mul(Nc, P1, 1, Gd, 0, tmp);        /* P1^+ G */
                        mat_mul(Nc, tmp, 0, P2, 1, X);         /* P1^+ G P2^+ */
                        cplx* Fl = Fo + ((size_t)z[i] * 4 + mu) * n2;
                        for (int e = 0; e < Nc * Nc; ++e) Fl[e] += X[e] / fact;
                    } else {
                        mat_mul(Nc, P2, 0, Gd, 1, tmp);        /* P2 G^+ */
                        mat_mul(Nc, tmp, 0, P1, 0, X);         /* P2 G^+ P1 */
                        cplx* Fl = Fo + ((size_t)z[i + 1] * 4 + mu) * n2;   /* V_mu(z_i - mu) */
                        for (int e = 0; e < Nc * Nc; ++e) Fl[e] += X[e] / fact;
                    }
                }
            }
        }
    }
    free(W81);
    free(G81);
}

/* Link gradient of L = Re <g, D psi> = Re sum_y g(y)^+ (D psi)(y), PyTorch's
 * convention F = dL/dRe V + i dL/dIm V.  Staggered, Wilson: a term
 * coef (S (x) C) with C = V contributes M^+ and one with C = V^+ contributes
 * M, with M of term_M.  Brillouin: through the paths of W (brillouin_force).
 * F is [site][mu][a][b]. */
int oracle_force(int op, int Nc, const int* L, int Nv, double mass, const real_t* V,
                 const real_t* psi, const real_t* g, real_t* F)
{
    if (Nc < 1 || Nc > MAX_NC) return 1;
    if (op == OP_BRILLOUIN) {
        ctx_t cb;
        set_ctx(&cb, op, Nc, L, Nv, mass, V, NULL);
        memset(F, 0, sizeof(cplx) * cb.vol * 4 * Nc * Nc);
        brillouin_force(&cb, (const cplx*)psi, (const cplx*)g, (cplx*)F);
        return 0;
    }
    ctx_t c;
    set_ctx(&c, op, Nc, L, Nv, mass, V, NULL);
    const cplx* P = (const cplx*)psi;
    const cplx* Gv = (const cplx*)g;
    cplx* Fo = (cplx*)F;
    memset(Fo, 0, sizeof(cplx) * c.vol * 4 * Nc * Nc);
    size_t blk = (size_t)Nv * c.Ns * Nc;
    term_t T[MAX_TERMS];
    cplx M[MAX_NC * MAX_NC];
    for (long y = 0; y < c.vol; ++y) {
        int nt = rows(&c, y, T, NULL);
        for (int t = 0; t < nt; ++t) {
            if (T[t].link_site < 0) continue;
            const cplx* py = P + blk * shift(&c, y, T[t].d);
            const cplx* gy = Gv + blk * y;
            for (int b = 0; b < Nc; ++b)
                for (int a = 0; a < Nc; ++a) {
                    cplx acc = 0;
                    for (int v = 0; v < Nv; ++v)
                        for (int s = 0; s < c.Ns; ++s)
                            for (int sp = 0; sp < c.Ns; ++sp) {
                                cplx Sv = (T[t].spin < 0) ? (s == sp ? 1.0 : 0.0) : G[T[t].spin][s][sp];
                                if (Sv == 0) continue;
                                acc += py[((size_t)v * c.Ns + sp) * Nc + b] * Sv *
                                       conj(gy[((size_t)v * c.Ns + s) * Nc + a]);
                            }
                    M[b * Nc + a] = T[t].coef * acc;
                }
            cplx* Fl = Fo + ((size_t)T[t].link_site * 4 + T[t].link_mu) * Nc * Nc;
            for (int a = 0; a < Nc; ++a)
                for (int b = 0; b < Nc; ++b)
                    Fl[a * Nc + b] += T[t].dag ? M[a * Nc + b] : conj(M[b * Nc + a]);
        }
    }
    return 0;
}

/* number of terms in one row (for the count pins) */
int oracle_row_terms(int op, int Nc, const int* L, double mass, const real_t* V, long y,
                     int* offsets /* [MAX_TERMS][4] or NULL */, int* spins /* or NULL */)
{
    ctx_t c;
    set_ctx(&c, op, Nc, L, 1, mass, V, NULL);
    term_t T[MAX_TERMS];
    cplx* W81buf = (op == OP_BRILLOUIN) ? malloc(sizeof(cplx) * 81 * Nc * Nc) : NULL;
    int n = rows(&c, y, T, W81buf);
    for (int t = 0; t < n; ++t) {
        if (offsets) memcpy(offsets + 4 * t, T[t].d, sizeof(int) * 4);
        if (spins) spins[t] = T[t].spin;
    }
    free(W81buf);
    return n;
}

int oracle_max_terms(void) { return MAX_TERMS; }
