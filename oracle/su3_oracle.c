/*
 * Plain CPU oracle for site-local lattice expression evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code;
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything is FP64, single-threaded, built without floating-point
 * contraction (-ffp-contract=off) so that x86-64 and aarch64 produce the same
 * bits.  Fields are in the canonical host layout:
 *   matrix  double[n][3][3][2]   (row i, column j, re/im)
 *   vector  double[n][3][2]
 *   real    double[n]
 * with n = volume * links; element m = site * links + mu.
 *
 * What is computed, with the passage of arXiv:1710.09409 it follows:
 *   oracle_mm      z = x*y for complex 3x3 matrices at every site: the
 *                  SU(3)xSU(3) streaming test (Sec. 4, Listing 3), written as
 *                  the definition z_ik = sum_j x_ij y_jk, j = 0,1,2 in order.
 *   oracle_mv      z = x*v, matrix times colour vector (same definition).
 *   oracle_eval    the value of an expression tree at every site, evaluated
 *                  recursively per site with per-site temporaries, as the
 *                  expression-template engine does (Sec. 3, Listing 1:
 *                  _odata[ss] = eval(ss, expr) for every ss).  Operators:
 *                  product, sum, difference, real scaling, Hermitian adjoint.
 *                  Real fields give Listing 2 (v3 = v1+v2, v3 = v1+v2+v1*v2).
 *   oracle_eval_adjoint  reverse-mode gradient of a real loss through the same
 *                  tree, per site (gradient convention dL/dRe + i dL/dIm).
 *   oracle_round   round to FP32 / BF16 / FP16 with round-to-nearest-even,
 *                  from the IEEE 754 definition (storage precisions).
 *   oracle_c12_expand  third row of a special unitary matrix rebuilt from the
 *                  first two: row2 = conj(row0 x row1).
 *   oracle_redot   sum over all reals of x*y (= sum_x Re tr(X^dagger Y)).
 *   oracle_reunitarize  Gram-Schmidt over rows and removal of the determinant
 *                  phase (principal cube root), in FP64.
 *   oracle_cshift  circular shift of a field along one lattice direction,
 *                  dst(x) = src(x + shift * e_dim) with periodic wrap (the
 *                  Cshift operation the paper names as the next step beside
 *                  its Dslash port, Sec. 6).
 *   oracle_hop     the colour part of the Wilson Dslash operator, the
 *                  nearest-neighbour hopping term of Sec. 6:
 *                  out(x) = sum_mu [ U_mu(x) v(x+mu) + U_mu(x-mu)^dagger v(x-mu) ],
 *                  v a colour vector or a colour matrix field, U the 4 links.
 *                  Site order: s = x + Lx*(y + Ly*(z + Lz*t)); directions
 *                  0..3 = x, y, z, t.
 *   oracle_dslash  the Wilson Dslash hopping term with its spin structure, the
 *                  operator whose port the paper names as its next step
 *                  (Sec. 6):
 *                  out(x) = sum_mu [ (1 - r gamma_mu) (x) U_mu(x) psi(x+mu)
 *                                  + (1 + r gamma_mu) (x) U_mu(x-mu)^dagger psi(x-mu) ],
 *                  psi a spinor field double[V][4][3][2] (spin, colour,
 *                  re/im), r = +1 for the operator (r = -1 swaps the two
 *                  projectors; the sum of both is twice the colour hopping
 *                  term on every spin).  Written as the plain definition: the
 *                  full 4x4 spin matrix (1 -+ r gamma_mu) applied to U psi.
 *                  Euclidean gamma matrices of the chiral basis,
 *                  gamma_5 = diag(1, 1, -1, -1) (oracle_gamma returns them).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

enum { OR_LEAF = 0, OR_MUL = 1, OR_ADD = 2, OR_SUB = 3, OR_SCALE = 4, OR_ADJ = 5 };
enum { OR_MATRIX = 0, OR_VECTOR = 1, OR_REAL = 2 };

typedef struct {
    int op;      /* OR_* */
    int a, b;    /* child node indices; children precede their parent */
    int leaf;    /* leaf slot (OR_LEAF) */
    double s;    /* real factor (OR_SCALE) */
} oracle_node;

static int width_of(int kind) { return kind == OR_MATRIX ? 18 : kind == OR_VECTOR ? 6 : 1; }

/* ---------- complex 3x3 helpers on interleaved re/im arrays ---------- */

/* z = x*y, x,y,z: 3x3 complex. z_ik = sum_j x_ij y_jk. */
static void mat_mul(const double* x, const double* y, double* z) {
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < 3; ++j) {
                double xr = x[2 * (3 * i + j)], xi = x[2 * (3 * i + j) + 1];
                double yr = y[2 * (3 * j + k)], yi = y[2 * (3 * j + k) + 1];
                re += xr * yr;
                re -= xi * yi;
                im += xr * yi;
                im += xi * yr;
            }
            z[2 * (3 * i + k)] = re;
            z[2 * (3 * i + k) + 1] = im;
        }
}

/* z = x*v, x: 3x3 complex, v: complex 3-vector. z_i = sum_j x_ij v_j. */
static void mat_vec(const double* x, const double* v, double* z) {
    for (int i = 0; i < 3; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 3; ++j) {
            double xr = x[2 * (3 * i + j)], xi = x[2 * (3 * i + j) + 1];
            double vr = v[2 * j], vi = v[2 * j + 1];
            re += xr * vr;
            re -= xi * vi;
            im += xr * vi;
            im += xi * vr;
        }
        z[2 * i] = re;
        z[2 * i + 1] = im;
    }
}

/* z = x^dagger (conjugate transpose). */
static void mat_adj(const double* x, double* z) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            z[2 * (3 * i + j)] = x[2 * (3 * j + i)];
            z[2 * (3 * i + j) + 1] = -x[2 * (3 * j + i) + 1];
        }
}

/* g = x * y^dagger for vectors x, y (outer product): g_ij = x_i conj(y_j). */
static void vec_outer_adj(const double* x, const double* y, double* g) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double xr = x[2 * i], xi = x[2 * i + 1], yr = y[2 * j], yi = y[2 * j + 1];
            g[2 * (3 * i + j)] = xr * yr + xi * yi;
            g[2 * (3 * i + j) + 1] = xi * yr - xr * yi;
        }
}

/* ---------- element-wise entry points ---------- */

void oracle_mm(const double* x, const double* y, double* z, int64_t n) {
    for (int64_t e = 0; e < n; ++e) mat_mul(x + 18 * e, y + 18 * e, z + 18 * e);
}

void oracle_mv(const double* x, const double* v, double* z, int64_t n) {
    for (int64_t e = 0; e < n; ++e) mat_vec(x + 18 * e, v + 6 * e, z + 6 * e);
}

/* ---------- expression trees ---------- */

#define MAXNODES 64

typedef struct { int kind; double v[18]; } value_t;

/* Kind of every node; returns 0, or -1 on a type error / malformed tree. */
static int infer_kinds(const oracle_node* nodes, int nnodes, const int* leaf_kind, int nleaves,
                       int* kind) {
    if (nnodes < 1 || nnodes > MAXNODES) return -1;
    for (int k = 0; k < nnodes; ++k) {
        const oracle_node* nd = &nodes[k];
        int ka = -1, kb = -1;
        if (nd->op != OR_LEAF) {
            if (nd->a < 0 || nd->a >= k) return -1;
            ka = kind[nd->a];
        }
        if (nd->op == OR_MUL || nd->op == OR_ADD || nd->op == OR_SUB) {
            if (nd->b < 0 || nd->b >= k) return -1;
            kb = kind[nd->b];
        }
        switch (nd->op) {
        case OR_LEAF:
            if (nd->leaf < 0 || nd->leaf >= nleaves) return -1;
            kind[k] = leaf_kind[nd->leaf];
            if (kind[k] < 0 || kind[k] > 2) return -1;
            break;
        case OR_MUL:
            if (ka == OR_MATRIX && kb == OR_MATRIX) kind[k] = OR_MATRIX;
            else if (ka == OR_MATRIX && kb == OR_VECTOR) kind[k] = OR_VECTOR;
            else if (ka == OR_REAL && kb == OR_REAL) kind[k] = OR_REAL;
            else return -1;
            break;
        case OR_ADD:
        case OR_SUB:
            if (ka != kb) return -1;
            kind[k] = ka;
            break;
        case OR_SCALE: kind[k] = ka; break;
        case OR_ADJ:
            if (ka != OR_MATRIX) return -1;
            kind[k] = OR_MATRIX;
            break;
        default: return -1;
        }
    }
    return 0;
}

/* Forward values of all nodes at element e. */
static void forward(const oracle_node* nodes, int nnodes, const int* kind,
                    const double* const* leaves, int64_t e, value_t* val) {
    for (int k = 0; k < nnodes; ++k) {
        const oracle_node* nd = &nodes[k];
        value_t* o = &val[k];
        o->kind = kind[k];
        int w = width_of(kind[k]);
        switch (nd->op) {
        case OR_LEAF: memcpy(o->v, leaves[nd->leaf] + (int64_t)w * e, sizeof(double) * w); break;
        case OR_MUL: {
            const value_t* x = &val[nd->a];
            const value_t* y = &val[nd->b];
            if (x->kind == OR_REAL) o->v[0] = x->v[0] * y->v[0];
            else if (y->kind == OR_VECTOR) mat_vec(x->v, y->v, o->v);
            else mat_mul(x->v, y->v, o->v);
            break;
        }
        case OR_ADD:
            for (int r = 0; r < w; ++r) o->v[r] = val[nd->a].v[r] + val[nd->b].v[r];
            break;
        case OR_SUB:
            for (int r = 0; r < w; ++r) o->v[r] = val[nd->a].v[r] - val[nd->b].v[r];
            break;
        case OR_SCALE:
            for (int r = 0; r < w; ++r) o->v[r] = nd->s * val[nd->a].v[r];
            break;
        case OR_ADJ: mat_adj(val[nd->a].v, o->v); break;
        }
    }
}

/* out[e] = value of node `root` at every element e < n.  Returns 0, -1 on a
 * malformed or ill-typed tree. */
int oracle_eval(const oracle_node* nodes, int nnodes, int root, const double* const* leaves,
                const int* leaf_kind, int nleaves, int64_t n, double* out) {
    int kind[MAXNODES];
    if (infer_kinds(nodes, nnodes, leaf_kind, nleaves, kind) != 0) return -1;
    if (root < 0 || root >= nnodes) return -1;
    int w = width_of(kind[root]);
    value_t val[MAXNODES];
    for (int64_t e = 0; e < n; ++e) {
        forward(nodes, root + 1, kind, leaves, e, val);
        memcpy(out + (int64_t)w * e, val[root].v, sizeof(double) * w);
    }
    return 0;
}

/* Reverse mode.  For a real loss L with dL/d(root) = gz (per element, in the
 * root's layout), accumulate dL/d(leaf slot) into gleaves[slot] (+=), for
 * every element.  Rules (gradient G of a node's value):
 *   Z = X*Y (matrices): dX += G Y^dagger, dY += X^dagger G
 *   Z = X*v:            dX += G v^dagger, dv += X^dagger G
 *   Z = x*y (reals):    dx += G y,        dy += x G
 *   Z = X+Y / X-Y:      dX += G,          dY += G / -G
 *   Z = s X:            dX += s G
 *   Z = X^dagger:       dX += G^dagger
 * Returns 0, -1 on a malformed tree. */
int oracle_eval_adjoint(const oracle_node* nodes, int nnodes, int root,
                        const double* const* leaves, const int* leaf_kind, int nleaves,
                        int64_t n, const double* gz, double* const* gleaves) {
    int kind[MAXNODES];
    if (infer_kinds(nodes, nnodes, leaf_kind, nleaves, kind) != 0) return -1;
    if (root < 0 || root >= nnodes) return -1;
    value_t val[MAXNODES], grad[MAXNODES];
    double t[18], u[18];
    for (int64_t e = 0; e < n; ++e) {
        forward(nodes, root + 1, kind, leaves, e, val);
        for (int k = 0; k <= root; ++k) memset(grad[k].v, 0, sizeof(grad[k].v));
        memcpy(grad[root].v, gz + (int64_t)width_of(kind[root]) * e, sizeof(double) * width_of(kind[root]));
        for (int k = root; k >= 0; --k) {
            const oracle_node* nd = &nodes[k];
            const double* G = grad[k].v;
            int w = width_of(kind[k]);
            switch (nd->op) {
            case OR_LEAF: {
                double* dst = gleaves[nd->leaf] + (int64_t)w * e;
                for (int r = 0; r < w; ++r) dst[r] += G[r];
                break;
            }
            case OR_MUL: {
                const value_t* x = &val[nd->a];
                const value_t* y = &val[nd->b];
                double* gx = grad[nd->a].v;
                double* gy = grad[nd->b].v;
                if (x->kind == OR_REAL) {
                    gx[0] += G[0] * y->v[0];
                    gy[0] += x->v[0] * G[0];
                } else if (y->kind == OR_VECTOR) {
                    vec_outer_adj(G, y->v, t);
                    for (int r = 0; r < 18; ++r) gx[r] += t[r];
                    mat_adj(x->v, u);
                    mat_vec(u, G, t);
                    for (int r = 0; r < 6; ++r) gy[r] += t[r];
                } else {
                    mat_adj(y->v, u);
                    mat_mul(G, u, t);
                    for (int r = 0; r < 18; ++r) gx[r] += t[r];
                    mat_adj(x->v, u);
                    mat_mul(u, G, t);
                    for (int r = 0; r < 18; ++r) gy[r] += t[r];
                }
                break;
            }
            case OR_ADD:
                for (int r = 0; r < w; ++r) { grad[nd->a].v[r] += G[r]; grad[nd->b].v[r] += G[r]; }
                break;
            case OR_SUB:
                for (int r = 0; r < w; ++r) { grad[nd->a].v[r] += G[r]; grad[nd->b].v[r] -= G[r]; }
                break;
            case OR_SCALE:
                for (int r = 0; r < w; ++r) grad[nd->a].v[r] += nd->s * G[r];
                break;
            case OR_ADJ:
                mat_adj(G, t);
                for (int r = 0; r < 18; ++r) grad[nd->a].v[r] += t[r];
                break;
            }
        }
    }
    return 0;
}

/* ---------- storage rounding (IEEE 754 round-to-nearest-even) ---------- */

/* Round x to a binary format with p significand bits (including the leading
 * one), minimum normal exponent emin and maximum exponent emax: the result is
 * q * 2^k with k = max(e - p, emin - p + 1), e the exponent of x with
 * x = m * 2^e, 0.5 <= |m| < 1, and q = x / 2^k rounded to the nearest integer,
 * ties to even (rint in the default rounding mode).  Results beyond the largest
 * finite value become infinities. */
static double round_format(double x, int p, int emin, int emax) {
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    int e;
    frexp(x, &e);
    int k = e - p;
    if (k < emin - p + 1) k = emin - p + 1;
    double q = rint(ldexp(x, -k));
    double r = ldexp(q, k);
    double maxfin = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
    if (fabs(r) > maxfin) return copysign(INFINITY, x);
    return r;
}

/* fmt: 0 = FP32 (p 24, emin -126, emax 127), 1 = BF16 (8, -126, 127),
 *      2 = FP16 (11, -14, 15).  Returns 0, -1 on an unknown format. */
int oracle_round(const double* in, double* out, int64_t n, int fmt) {
    int p, emin, emax;
    switch (fmt) {
    case 0: p = 24; emin = -126; emax = 127; break;
    case 1: p = 8; emin = -126; emax = 127; break;
    case 2: p = 11; emin = -14; emax = 15; break;
    default: return -1;
    }
    for (int64_t i = 0; i < n; ++i) out[i] = round_format(in[i], p, emin, emax);
    return 0;
}

/* ---------- two-row (12-real) storage of special unitary matrices ---------- */

/* full[e] = the 3x3 matrix whose rows 0 and 1 are rows01[e] ([2][3][2]) and
 * whose row 2 is conj(row0 x row1):
 *   r2_0 = conj(r0_1 r1_2 - r0_2 r1_1)
 *   r2_1 = conj(r0_2 r1_0 - r0_0 r1_2)
 *   r2_2 = conj(r0_0 r1_1 - r0_1 r1_0)                                    */
void oracle_c12_expand(const double* rows01, double* full, int64_t n) {
    for (int64_t e = 0; e < n; ++e) {
        const double* r = rows01 + 12 * e;
        double* f = full + 18 * e;
        memcpy(f, r, sizeof(double) * 12);
        for (int c = 0; c < 3; ++c) {
            int j = (c + 1) % 3, k = (c + 2) % 3;
            double ar = r[2 * j], ai = r[2 * j + 1];           /* r0_j */
            double br = r[6 + 2 * k], bi = r[6 + 2 * k + 1];   /* r1_k */
            double cr = r[2 * k], ci = r[2 * k + 1];           /* r0_k */
            double dr = r[6 + 2 * j], di = r[6 + 2 * j + 1];   /* r1_j */
            double re = (ar * br - ai * bi) - (cr * dr - ci * di);
            double im = (ar * bi + ai * br) - (cr * di + ci * dr);
            f[12 + 2 * c] = re;
            f[12 + 2 * c + 1] = -im;
        }
    }
}

/* ---------- reductions ---------- */

/* sum_i x_i y_i over n reals, in index order. */
double oracle_redot(const double* x, const double* y, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* ---------- projection back to SU(3) ---------- */

/* out[e] = SU(3) matrix from in[e]: rows orthonormalised by modified
 * Gram-Schmidt (row 0, then row 1 against row 0, then row 2 against rows 0 and
 * 1, each projection sweep done twice), then multiplied by exp(-i phi/3) with
 * phi = arg det, principal branch (-pi, pi]. */
void oracle_reunitarize(const double* in, double* out, int64_t n) {
    for (int64_t e = 0; e < n; ++e) {
        double r[18];
        memcpy(r, in + 18 * e, sizeof r);
        for (int i = 0; i < 3; ++i) {
            for (int rep = 0; rep < 2; ++rep)
                for (int p = 0; p < i; ++p) {
                    double cr = 0.0, ci = 0.0;          /* <r_p, r_i> = sum conj(r_p) r_i */
                    for (int j = 0; j < 3; ++j) {
                        double pr = r[6 * p + 2 * j], pi = r[6 * p + 2 * j + 1];
                        double xr = r[6 * i + 2 * j], xi = r[6 * i + 2 * j + 1];
                        cr += pr * xr + pi * xi;
                        ci += pr * xi - pi * xr;
                    }
                    for (int j = 0; j < 3; ++j) {
                        double pr = r[6 * p + 2 * j], pi = r[6 * p + 2 * j + 1];
                        r[6 * i + 2 * j] -= cr * pr - ci * pi;
                        r[6 * i + 2 * j + 1] -= cr * pi + ci * pr;
                    }
                }
            double nn = 0.0;
            for (int j = 0; j < 6; ++j) nn += r[6 * i + j] * r[6 * i + j];
            double inv = 1.0 / sqrt(nn);
            for (int j = 0; j < 6; ++j) r[6 * i + j] *= inv;
        }
        /* det = sum_j r0_j * cof_j, cof_j = r1_{j+1} r2_{j+2} - r1_{j+2} r2_{j+1} */
        double dr = 0.0, di = 0.0;
        for (int j = 0; j < 3; ++j) {
            int a = (j + 1) % 3, b = (j + 2) % 3;
            double xr = r[6 + 2 * a] * r[12 + 2 * b] - r[6 + 2 * a + 1] * r[12 + 2 * b + 1]
                      - (r[6 + 2 * b] * r[12 + 2 * a] - r[6 + 2 * b + 1] * r[12 + 2 * a + 1]);
            double xi = r[6 + 2 * a] * r[12 + 2 * b + 1] + r[6 + 2 * a + 1] * r[12 + 2 * b]
                      - (r[6 + 2 * b] * r[12 + 2 * a + 1] + r[6 + 2 * b + 1] * r[12 + 2 * a]);
            dr += r[2 * j] * xr - r[2 * j + 1] * xi;
            di += r[2 * j] * xi + r[2 * j + 1] * xr;
        }
        double phi = atan2(di, dr);
        double c = cos(-phi / 3.0), s = sin(-phi / 3.0);
        double* o = out + 18 * e;
        for (int q = 0; q < 9; ++q) {
            o[2 * q] = c * r[2 * q] - s * r[2 * q + 1];
            o[2 * q + 1] = c * r[2 * q + 1] + s * r[2 * q];
        }
    }
}

/* ---------- neighbours: Cshift and the hopping term ---------- */

/* site index of (x,y,z,t) + shift * e_dim, periodic */
static int64_t shifted_site(int64_t s, const int* L, int dim, int shift) {
    int64_t c[4];
    int64_t r = s;
    for (int d = 0; d < 4; ++d) {
        c[d] = r % L[d];
        r /= L[d];
    }
    int64_t m = ((c[dim] + shift) % L[dim] + L[dim]) % L[dim];
    c[dim] = m;
    return c[0] + (int64_t)L[0] * (c[1] + (int64_t)L[1] * (c[2] + (int64_t)L[2] * c[3]));
}

/* dst(x) = src(x + shift e_dim); `width` doubles per site (all links and
 * components of the site). */
void oracle_cshift(const double* src, double* dst, const int* L, int width, int dim, int shift) {
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    for (int64_t s = 0; s < V; ++s) {
        const int64_t n = shifted_site(s, L, dim, shift);
        memcpy(dst + width * s, src + width * n, sizeof(double) * (size_t)width);
    }
}

/* out(x) = sum_mu U_mu(x) v(x+mu) + U_mu(x-mu)^dagger v(x-mu); U: 4 links per
 * site (double[V][4][3][3][2]); v, out: matrix (kind 0) or vector (kind 1). */
void oracle_hop(const double* U, const double* v, double* out, const int* L, int kind) {
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    const int w = width_of(kind);
    double t[18], a[18];
    for (int64_t s = 0; s < V; ++s) {
        double* o = out + w * s;
        for (int r = 0; r < w; ++r) o[r] = 0.0;
        for (int mu = 0; mu < 4; ++mu) {
            const int64_t fw = shifted_site(s, L, mu, +1);
            const int64_t bw = shifted_site(s, L, mu, -1);
            /* forward: U_mu(x) v(x+mu) */
            if (kind == OR_MATRIX) mat_mul(U + 18 * (4 * s + mu), v + w * fw, t);
            else mat_vec(U + 18 * (4 * s + mu), v + w * fw, t);
            for (int r = 0; r < w; ++r) o[r] += t[r];
            /* backward: U_mu(x-mu)^dagger v(x-mu) */
            mat_adj(U + 18 * (4 * bw + mu), a);
            if (kind == OR_MATRIX) mat_mul(a, v + w * bw, t);
            else mat_vec(a, v + w * bw, t);
            for (int r = 0; r < w; ++r) o[r] += t[r];
        }
    }
}

/* ---------- the Wilson hopping term with spin ---------- */

/* Euclidean gamma matrices, chiral basis: gamma_mu = [[0, s_mu], [s_mu^+, 0]]
 * in 2x2 spin blocks, s_x = [[0, i], [i, 0]], s_y = [[0, -1], [1, 0]],
 * s_z = [[i, 0], [0, -i]], s_t = identity; entry [mu][row][col][re/im].
 * Index 4 is gamma_5 = diag(1, 1, -1, -1). */
static const double GAMMA[5][4][4][2] = {
    {{{0, 0}, {0, 0}, {0, 0}, {0, 1}},
     {{0, 0}, {0, 0}, {0, 1}, {0, 0}},
     {{0, 0}, {0, -1}, {0, 0}, {0, 0}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}},
     {{0, 0}, {0, 0}, {1, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}},
     {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 1}, {0, 0}},
     {{0, 0}, {0, 0}, {0, 0}, {0, -1}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {1, 0}, {0, 0}},
     {{0, 0}, {0, 0}, {0, 0}, {1, 0}},
     {{1, 0}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}}},
    {{{1, 0}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {0, 0}, {-1, 0}, {0, 0}},
     {{0, 0}, {0, 0}, {0, 0}, {-1, 0}}},
};

/* gamma_mu (mu = 0..3) or gamma_5 (mu = 4) as double[4][4][2]; -1 for a bad mu. */
int oracle_gamma(int mu, double* out) {
    if (mu < 0 || mu > 4) return -1;
    memcpy(out, GAMMA[mu], sizeof GAMMA[mu]);
    return 0;
}

/* o (spinor, 24 doubles) += P chi, P = 1 + sg * r * gamma_mu (4x4 complex),
 * chi[s] = the colour vector of spin s (already multiplied by the link). */
static void spin_project_add(double* o, const double chi[4][6], int mu, double sgr) {
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double pr = sgr * GAMMA[mu][a][b][0], pi = sgr * GAMMA[mu][a][b][1];
            if (a == b) pr += 1.0;
            for (int c = 0; c < 3; ++c) {
                double xr = chi[b][2 * c], xi = chi[b][2 * c + 1];
                o[6 * a + 2 * c] += pr * xr;
                o[6 * a + 2 * c] -= pi * xi;
                o[6 * a + 2 * c + 1] += pr * xi;
                o[6 * a + 2 * c + 1] += pi * xr;
            }
        }
}

/* out(x) = sum_mu (1 - r g_mu) U_mu(x) psi(x+mu) + (1 + r g_mu) U_mu(x-mu)^+ psi(x-mu);
 * U: double[V][4][3][3][2]; psi, out: double[V][4][3][2]. */
void oracle_dslash(const double* U, const double* psi, double* out, const int* L, int r) {
    const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
    double chi[4][6], a[18];
    for (int64_t s = 0; s < V; ++s) {
        double* o = out + 24 * s;
        for (int k = 0; k < 24; ++k) o[k] = 0.0;
        for (int mu = 0; mu < 4; ++mu) {
            const int64_t fw = shifted_site(s, L, mu, +1);
            const int64_t bw = shifted_site(s, L, mu, -1);
            for (int sp = 0; sp < 4; ++sp) mat_vec(U + 18 * (4 * s + mu), psi + 24 * fw + 6 * sp, chi[sp]);
            spin_project_add(o, (const double(*)[6])chi, mu, -(double)r);
            mat_adj(U + 18 * (4 * bw + mu), a);
            for (int sp = 0; sp < 4; ++sp) mat_vec(a, psi + 24 * bw + 6 * sp, chi[sp]);
            spin_project_add(o, (const double(*)[6])chi, mu, (double)r);
        }
    }
}
