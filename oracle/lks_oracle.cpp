/*
 * Plain, single-threaded CPU oracle for the lattice kinetic scheme (LKS) with Brinkman
 * penalisation, the rigid-motion transfer from the design grid, the time-averaged objective
 * and its exact discrete adjoint (arXiv 2506.23895, Secs. 2.2-2.5, Algorithms 1 and 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm do.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Arithmetic is IEEE double (the scalar template is also instantiated with
 * std::complex<double> for complex-step differentiation).  Every loop runs in the order the
 * definitions state; nothing is blocked, fused or reordered.  Readings of points the paper
 * leaves open are marked "reading:" below.
 *
 * Pins (tests/test_oracle_*.py): shear-wave decay factor (exact solution of the discrete
 * scheme), plane Poiseuille and Couette profiles as exact fixed points, mass conservation in a
 * periodic box, uniform-flow invariance, hand-computed transfer weights, partition of unity,
 * rotation direction, complex-step and central-difference checks of the adjoint gradient.
 */
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

typedef std::complex<double> cplx;

// ----------------------------------------------------------------- lattice (Sec. 2.2)
// D2Q9 for 2D and D3Q15 for 3D.  The velocity figure is missing from the paper; the sets and
// weights are the standard ones (rest 4/9, axes 1/9, diagonals 1/36 for D2Q9; rest 2/9,
// axes 1/9, cube corners 1/72 for D3Q15).
struct Lattice {
    int Q;
    int c[15][3];
    double w[15];
};

Lattice make_lattice(int dim) {
    Lattice L;
    std::memset(&L, 0, sizeof(L));
    if (dim == 2) {
        const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
        L.Q = 9;
        for (int i = 0; i < 9; ++i) {
            L.c[i][0] = c[i][0];
            L.c[i][1] = c[i][1];
            L.c[i][2] = 0;
            L.w[i] = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else {
        const int c[15][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                              {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
        L.Q = 15;
        for (int i = 0; i < 15; ++i) {
            for (int a = 0; a < 3; ++a) L.c[i][a] = c[i][a];
            L.w[i] = (i == 0) ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
        }
    }
    return L;
}

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3 };

}  // namespace

extern "C" {

/* Problem statement handed in by the tests (mirrors workloads.Problem field by field). */
typedef struct {
    int dim, nx, ny, nz, lx, ly, lz;
    double A, kappa_max, q, rho0;
    int bc[6];
    double bc_val[6][4]; /* ux, uy, uz, rho */
    double u_init[3], body_force[3], xi_G[3];
    int obj_kind;
    int obj_box[6];
    double obj_dir[3];
    double obj_cyl_r, obj_cyl_c[2];
    int win_begin, win_end;
    double rot_axis[3]; /* 3D rotation axis (unit vector); (0, 0, 1) or all zero: the z axis */
} orc_problem;

}  // extern "C"

namespace {

std::string g_err;

struct Grid {
    int dim, n[3];
    bool periodic[3];  // per axis; inactive axes (z in 2D) count as periodic of extent 1
    long nodes;
    long idx(int x, int y, int z) const { return ((long)z * n[1] + y) * n[0] + x; }
};

Grid make_grid(const orc_problem& p) {
    Grid g;
    g.dim = p.dim;
    g.n[0] = p.nx;
    g.n[1] = p.ny;
    g.n[2] = (p.dim == 2) ? 1 : p.nz;
    for (int a = 0; a < 3; ++a) g.periodic[a] = (a >= p.dim) || (p.bc[2 * a] == BC_PERIODIC);
    g.nodes = (long)g.n[0] * g.n[1] * g.n[2];
    return g;
}

int wrap(int i, int n) { return ((i % n) + n) % n; }

bool on_boundary(const Grid& g, const int x[3]) {
    for (int a = 0; a < g.dim; ++a)
        if (!g.periodic[a] && (x[a] == 0 || x[a] == g.n[a] - 1)) return true;
    return false;
}

// reading (the paper prescribes rho or u on boundary nodes but not the unprescribed
// quantity): boundary nodes copy the rest from the interior node one step inward along every
// boundary normal they lie on; WALL beats INLET beats OUTLET on edges and corners, ties go to
// the lower face index.
int precedence(int t) { return t == BC_WALL ? 3 : (t == BC_INLET ? 2 : (t == BC_OUTLET ? 1 : 0)); }

int winning_face(const orc_problem& p, const Grid& g, const int x[3]) {
    int best = -1;
    for (int a = 0; a < g.dim; ++a) {
        if (g.periodic[a]) continue;
        int f = -1;
        if (x[a] == 0) f = 2 * a;
        else if (x[a] == g.n[a] - 1) f = 2 * a + 1;
        if (f < 0) continue;
        if (best < 0 || precedence(p.bc[f]) > precedence(p.bc[best])) best = f;
    }
    return best;
}

void inward(const Grid& g, const int x[3], int s[3]) {
    for (int a = 0; a < 3; ++a) {
        s[a] = x[a];
        if (a < g.dim && !g.periodic[a]) {
            if (x[a] == 0) s[a] = 1;
            else if (x[a] == g.n[a] - 1) s[a] = g.n[a] - 2;
        }
    }
}

// One first-derivative operator per axis (reading: the paper does not say how the velocity
// gradient in f^eq is discretised): second-order central difference, periodic wrap, and the
// second-order one-sided difference along the normal on a non-periodic boundary node.
// Returns the taps (offset along the axis, coefficient) used at coordinate i.
int deriv_taps(const Grid& g, int axis, int i, int off[3], double coef[3]) {
    int n = g.n[axis];
    if (g.periodic[axis]) {
        off[0] = +1; coef[0] = 0.5;
        off[1] = -1; coef[1] = -0.5;
        return 2;
    }
    if (i == 0) {
        off[0] = 0; coef[0] = -1.5;
        off[1] = 1; coef[1] = 2.0;
        off[2] = 2; coef[2] = -0.5;
        return 3;
    }
    if (i == n - 1) {
        off[0] = 0; coef[0] = 1.5;
        off[1] = -1; coef[1] = -2.0;
        off[2] = -2; coef[2] = 0.5;
        return 3;
    }
    off[0] = +1; coef[0] = 0.5;
    off[1] = -1; coef[1] = -0.5;
    return 2;
}

template <class T>
struct State {
    std::vector<T> rho, u[3];
    void resize(long n) {
        rho.assign(n, T(0));
        for (int a = 0; a < 3; ++a) u[a].assign(n, T(0));
    }
};

// ----------------------------------------------------------------- transfer (Sec. 2.3)

// Peskin's four-point cosine kernel (Sec. 2.3, weight function w).  Reading: the printed
// "1 - cos" is a typesetting slip; 1 + cos is the kernel of the cited reference and is the
// one whose integer-shifted copies sum to one.
double peskin_w(double r) {
    double a = std::fabs(r);
    if (a >= 2.0) return 0.0;
    return 0.25 * (1.0 + std::cos(M_PI * r / 2.0));
}

template <class T>
T kappa_ref(const orc_problem& p, T gamma) {
    // Brinkman coefficient interpolation (Sec. 2.3): kappa_max * q*gamma / ((1-gamma) + q)
    return p.kappa_max * p.q * gamma / ((1.0 - gamma) + p.q);
}

double kappa_ref_prime(const orc_problem& p, double gamma) {
    double d = (1.0 - gamma) + p.q;
    return p.kappa_max * p.q * (1.0 + p.q) / (d * d);
}

// True when a 3D problem rotates about an axis other than z.
bool general_axis(const orc_problem& p) {
    const double* a = p.rot_axis;
    return p.dim == 3 && !(a[0] == 0.0 && a[1] == 0.0 && (a[2] == 0.0 || a[2] == 1.0));
}

// Position and velocity of design node xi (Eqs. rigid_body_position / rigid_body_velocity).
// In 2D the rotation is in the plane; in 3D about the z axis (the 3D rotor of Sec. 3.3) or,
// for a general unit axis a, by Rodrigues' formula R = cos(th) I + sin(th) [a]x +
// (1 - cos(th)) a a^T, whose time derivative gives u_ref = omega a x (R (xi - xi_G)) + u_G.
void rigid_point(const orc_problem& p, const double* mrow, const int xi[3], double xr[3],
                 double ur[3]) {
    double th = mrow[0], om = mrow[1];
    const double* xG = mrow + 2;
    const double* uG = mrow + 5;
    double dx = xi[0] - p.xi_G[0], dy = xi[1] - p.xi_G[1], dz = xi[2] - p.xi_G[2];
    double c = std::cos(th), s = std::sin(th);
    if (general_axis(p)) {
        const double* a = p.rot_axis;
        const double d[3] = {dx, dy, dz};
        const double ad = a[0] * dx + a[1] * dy + a[2] * dz;
        const double axd[3] = {a[1] * dz - a[2] * dy, a[2] * dx - a[0] * dz, a[0] * dy - a[1] * dx};
        double rd[3];
        for (int k = 0; k < 3; ++k) rd[k] = c * d[k] + s * axd[k] + (1.0 - c) * a[k] * ad;
        const double w[3] = {a[1] * rd[2] - a[2] * rd[1], a[2] * rd[0] - a[0] * rd[2],
                             a[0] * rd[1] - a[1] * rd[0]};
        for (int k = 0; k < 3; ++k) {
            xr[k] = rd[k] + xG[k];
            ur[k] = om * w[k] + uG[k];
        }
        return;
    }
    xr[0] = c * dx - s * dy + xG[0];
    xr[1] = s * dx + c * dy + xG[1];
    ur[0] = (-s * dx - c * dy) * om + uG[0];
    ur[1] = (c * dx - s * dy) * om + uG[1];
    if (p.dim == 3) {
        xr[2] = dz + xG[2];
        ur[2] = uG[2];
    } else {
        xr[2] = 0.0;
        ur[2] = 0.0;
    }
}

// kappa(x) = sum_xi W(x - x_ref(xi)) kappa_ref(xi),  u_S(x) = sum_xi W u_ref(xi)
// (Eqs. brinkman_ref, velocity_ref; the integral over D is the sum over design nodes with
// unit cell volume).  Done by the definition: every design node scatters onto every analysis
// node inside its kernel support.
template <class T>
bool transfer(const orc_problem& p, const Grid& g, const std::vector<T>& kref,
              const double* mrow, std::vector<T>& kappa, std::vector<double> us[3]) {
    kappa.assign(g.nodes, T(0));
    for (int a = 0; a < 3; ++a) us[a].assign(g.nodes, 0.0);
    if (p.lx <= 0) return true;
    int lz = (p.dim == 2) ? 1 : p.lz;
    for (int k = 0; k < lz; ++k)
        for (int j = 0; j < p.ly; ++j)
            for (int i = 0; i < p.lx; ++i) {
                int xi[3] = {i, j, k};
                double xr[3], ur[3];
                rigid_point(p, mrow, xi, xr, ur);
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    if (a < p.dim) {
                        lo[a] = (int)std::floor(xr[a]) - 1;
                        hi[a] = (int)std::floor(xr[a]) + 2;
                    } else {
                        lo[a] = hi[a] = 0;
                    }
                }
                long dn = ((long)k * p.ly + j) * p.lx + i;
                for (int z = lo[2]; z <= hi[2]; ++z)
                    for (int y = lo[1]; y <= hi[1]; ++y)
                        for (int x = lo[0]; x <= hi[0]; ++x) {
                            int xa[3] = {x, y, z};
                            double W = 1.0;
                            for (int a = 0; a < p.dim; ++a) W *= peskin_w(xa[a] - xr[a]);
                            if (W == 0.0) continue;
                            // the support must lie inside the grid and off the boundary layer
                            for (int a = 0; a < p.dim; ++a) {
                                if (xa[a] < 0 || xa[a] >= g.n[a]) {
                                    g_err = "design footprint leaves the analysis grid";
                                    return false;
                                }
                            }
                            if (on_boundary(g, xa)) {
                                g_err = "design footprint touches a boundary node";
                                return false;
                            }
                            long n = g.idx(x, y, z);
                            kappa[n] += W * kref[dn];
                            for (int a = 0; a < 3; ++a) us[a][n] += W * ur[a];
                        }
            }
    return true;
}

// Transpose of the kappa part of the transfer, applied to a field e on the analysis grid:
// out(xi) = sum_x W(x - x_ref(xi)) e(x).
void transfer_T(const orc_problem& p, const Grid& g, const double* mrow,
                const std::vector<double>& e, std::vector<double>& out) {
    int lz = (p.dim == 2) ? 1 : p.lz;
    out.assign((long)p.lx * p.ly * lz, 0.0);
    for (int k = 0; k < lz; ++k)
        for (int j = 0; j < p.ly; ++j)
            for (int i = 0; i < p.lx; ++i) {
                int xi[3] = {i, j, k};
                double xr[3], ur[3];
                rigid_point(p, mrow, xi, xr, ur);
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    if (a < p.dim) {
                        lo[a] = (int)std::floor(xr[a]) - 1;
                        hi[a] = (int)std::floor(xr[a]) + 2;
                    } else {
                        lo[a] = hi[a] = 0;
                    }
                }
                double acc = 0.0;
                for (int z = lo[2]; z <= hi[2]; ++z)
                    for (int y = lo[1]; y <= hi[1]; ++y)
                        for (int x = lo[0]; x <= hi[0]; ++x) {
                            int xa[3] = {x, y, z};
                            double W = 1.0;
                            for (int a = 0; a < p.dim; ++a) W *= peskin_w(xa[a] - xr[a]);
                            if (W == 0.0) continue;
                            acc += W * e[g.idx(x, y, z)];
                        }
                out[((long)k * p.ly + j) * p.lx + i] = acc;
            }
}

// ----------------------------------------------------------------- objective (Sec. 2.5)

bool in_target(const orc_problem& p, int x, int y, int z) {
    const int* b = p.obj_box;
    if (x < b[0] || x > b[1] || y < b[2] || y > b[3]) return false;
    if (p.dim == 3 && (z < b[4] || z > b[5])) return false;
    if (p.obj_cyl_r > 0.0) {
        double dx = x - p.obj_cyl_c[0], dy = y - p.obj_cyl_c[1];
        if (dx * dx + dy * dy > p.obj_cyl_r * p.obj_cyl_r) return false;
    }
    return true;
}

long target_count(const orc_problem& p, const Grid& g) {
    long c = 0;
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) c += in_target(p, x, y, z) ? 1 : 0;
    return c;
}

// j(s) for one time level: J1 = -mean pressure (p = rho/3), J2 = -mean of n.u over the region.
template <class T>
T objective_level(const orc_problem& p, const Grid& g, const State<T>& s, long count) {
    T acc = T(0);
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                if (!in_target(p, x, y, z)) continue;
                long n = g.idx(x, y, z);
                if (p.obj_kind == 0) {
                    acc += s.rho[n] / 3.0;
                } else {
                    for (int a = 0; a < 3; ++a) acc += p.obj_dir[a] * s.u[a][n];
                }
            }
    return -acc / (double)count;
}

// ----------------------------------------------------------------- forward step (Alg. 1)

template <class T>
struct Solver {
    orc_problem p;
    Grid g;
    Lattice L;
    std::vector<T> kref;
    std::vector<double> gamma;
    std::vector<double> ks;   // static Brinkman coefficient per analysis node (empty: none)
    const double* motion;
    long count;

    bool init(const orc_problem& pp, const double* gam, const double* mot) {
        p = pp;
        g = make_grid(p);
        L = make_lattice(p.dim);
        motion = mot;
        for (int a = 0; a < p.dim; ++a)
            if (g.n[a] < 3) {
                g_err = "every active axis needs at least 3 nodes";
                return false;
            }
        if (p.dim == 3 && (!g.periodic[2] && g.n[2] < 3)) return false;
        long dn = (p.lx > 0) ? (long)p.lx * p.ly * ((p.dim == 2) ? 1 : p.lz) : 0;
        gamma.assign(gam, gam + dn);
        kref.assign(dn, T(0));
        count = target_count(p, g);
        if (count == 0) {
            g_err = "objective region is empty";
            return false;
        }
        return true;
    }

    void set_kref_complex(const double* dir, double h);

    void initial(State<T>& s, const double* init) {
        s.resize(g.nodes);
        for (long n = 0; n < g.nodes; ++n) {
            if (init) {
                s.rho[n] = init[n];
                for (int a = 0; a < 3; ++a) s.u[a][n] = init[(1 + a) * g.nodes + n];
            } else {
                s.rho[n] = p.rho0;
                for (int a = 0; a < 3; ++a) s.u[a][n] = p.u_init[a];
            }
        }
        if (!init) apply_bc(s);
    }

    // Macroscopic boundary conditions (Eqs. bc_rho, bc_u) on every boundary node.
    void apply_bc(State<T>& s) {
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    int xa[3] = {x, y, z};
                    if (!on_boundary(g, xa)) continue;
                    int f = winning_face(p, g, xa);
                    int sx[3];
                    inward(g, xa, sx);
                    long b = g.idx(x, y, z), src = g.idx(sx[0], sx[1], sx[2]);
                    int t = p.bc[f];
                    if (t == BC_WALL || t == BC_INLET) {
                        for (int a = 0; a < 3; ++a) s.u[a][b] = p.bc_val[f][a];
                        s.rho[b] = s.rho[src];
                    } else {  // outlet: rho and tangential u prescribed, normal u copied
                        int na = f / 2;
                        s.rho[b] = p.bc_val[f][3];
                        for (int a = 0; a < 3; ++a)
                            s.u[a][b] = (a == na) ? s.u[a][src] : T(p.bc_val[f][a]);
                    }
                }
    }

    // velocity-gradient tensor component d u_alpha / d x_beta at node (x,y,z)
    T grad(const State<T>& s, int alpha, int beta, const int xa[3]) {
        int off[3];
        double coef[3];
        int nt = deriv_taps(g, beta, xa[beta], off, coef);
        T acc = T(0);
        for (int t = 0; t < nt; ++t) {
            int xb[3] = {xa[0], xa[1], xa[2]};
            xb[beta] = wrap(xa[beta] + off[t], g.n[beta]);
            acc += coef[t] * s.u[alpha][g.idx(xb[0], xb[1], xb[2])];
        }
        return acc;
    }

    // One step s^{n-1} -> s^n at t_n (Alg. 1).  Stores kappa^n, u_S^n for the caller.
    bool step(const State<T>& s, State<T>& out, int n, std::vector<T>& kappa,
              std::vector<double> us[3]) {
        const int Q = L.Q, d = p.dim;
        // f_i^eq at every node from the old state (Sec. 2.2, equilibrium with the A term)
        std::vector<T> F((size_t)Q * g.nodes);
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    int xa[3] = {x, y, z};
                    long m = g.idx(x, y, z);
                    T S[3][3];
                    for (int al = 0; al < 3; ++al)
                        for (int be = 0; be < 3; ++be) S[al][be] = T(0);
                    for (int al = 0; al < d; ++al)
                        for (int be = 0; be < d; ++be) {
                            S[al][be] += grad(s, al, be, xa);
                            S[be][al] += grad(s, al, be, xa);
                        }
                    T uu = T(0);
                    for (int a = 0; a < d; ++a) uu += s.u[a][m] * s.u[a][m];
                    for (int i = 0; i < Q; ++i) {
                        T cu = T(0);
                        for (int a = 0; a < d; ++a) cu += (double)L.c[i][a] * s.u[a][m];
                        T cSc = T(0);
                        for (int al = 0; al < d; ++al)
                            for (int be = 0; be < d; ++be)
                                cSc += (double)(L.c[i][al] * L.c[i][be]) * S[al][be];
                        F[(size_t)i * g.nodes + m] =
                            L.w[i] * (s.rho[m] + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu + p.A * cSc);
                    }
                }
        // motion first, then the transfer (Alg. 1 order)
        const double* mrow = motion + 8 * (long)n;
        if (!transfer(p, g, kref, mrow, kappa, us)) return false;
        out.resize(g.nodes);
        // rho* and u* gathered from x - c_i (Eqs. rho, u), then the Brinkman force (Eq. u_ex_2)
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    int xa[3] = {x, y, z};
                    if (on_boundary(g, xa)) continue;
                    long m = g.idx(x, y, z);
                    T rs = T(0), us_[3] = {T(0), T(0), T(0)};
                    for (int i = 0; i < Q; ++i) {
                        int xs = wrap(x - L.c[i][0], g.n[0]);
                        int ys = wrap(y - L.c[i][1], g.n[1]);
                        int zs = wrap(z - L.c[i][2], g.n[2]);
                        T f = F[(size_t)i * g.nodes + g.idx(xs, ys, zs)];
                        rs += f;
                        for (int a = 0; a < d; ++a) us_[a] += (double)L.c[i][a] * f;
                    }
                    out.rho[m] = rs;
                    T k = kappa[m];
                    // implicit Brinkman update (Eq. u_ex_2); a static solid adds kappa_s with
                    // zero solid velocity to the denominator
                    const double kst = ks.empty() ? 0.0 : ks[m];
                    for (int a = 0; a < 3; ++a)
                        out.u[a][m] = (us_[a] + p.body_force[a] + k * us[a][m]) / (1.0 + k + kst);
                    if (d == 2) out.u[2][m] = T(0);
                }
        apply_bc(out);
        return true;
    }

    bool forward(int N, const double* init, T& J, std::vector<State<T>>* hist, State<T>& fin,
                 const double* lam_term = nullptr) {
        State<T> s, t;
        initial(s, init);
        if (hist) {
            hist->clear();
            hist->push_back(s);
        }
        J = T(0);
        double h = 1.0 / (double)(p.win_end - p.win_begin + 1);
        std::vector<T> kappa;
        std::vector<double> us[3];
        for (int n = 1; n <= N; ++n) {
            if (!step(s, t, n, kappa, us)) return false;
            std::swap(s, t);
            if (n >= p.win_begin && n <= p.win_end) J += h * objective_level(p, g, s, count);
            if (hist) hist->push_back(s);
        }
        fin = s;
        if (lam_term)   // terminal term <lam_term, s^N> of an augmented objective
            for (long m = 0; m < g.nodes; ++m) {
                J += lam_term[m] * s.rho[m];
                for (int a = 0; a < 3; ++a) J += lam_term[(1 + a) * g.nodes + m] * s.u[a][m];
            }
        return true;
    }
};

template <>
void Solver<cplx>::set_kref_complex(const double* dir, double h) {
    for (size_t k = 0; k < kref.size(); ++k)
        kref[k] = kappa_ref<cplx>(p, cplx(gamma[k], h * (dir ? dir[k] : 0.0)));
}

template <class T>
void set_kref_real(Solver<T>& S) {
    for (size_t k = 0; k < S.kref.size(); ++k) S.kref[k] = kappa_ref<double>(S.p, S.gamma[k]);
}

// ----------------------------------------------------------------- exact discrete adjoint
// Reverse sweep of the forward steps (the structure of Alg. 2): lambda^n = dJ/ds^n.  For
// n = N..1: add the objective's direct term at level n, push boundary-node adjoints back onto
// the interior nodes they were copied from (transpose of Eqs. bc_rho / bc_u), divide the
// velocity part by (1+kappa) (transpose of Eq. u_ex_2), accumulate the design sensitivity
// through the transposed transfer (Sec. 2.4, J' = sum 3 kappa'(u - u_S) u~ in the paper's
// form, here with the exact factor), then transpose the gather and the equilibrium
// (Eqs. arho, au, as and the adjoint equilibrium) including the transposed gradient stencil.
// paper = true follows Sec. 2.4's source update as printed instead: the (1 + kappa)^-1 of the
// Brinkman source (Eq. au_ex) divides only the gathered first moment 3 U~ and the objective
// source, not the whole adjoint velocity.  (Boundary values keep the transposed copies: with a
// boundary objective such as J1, dropping them would discard the whole sensitivity.)
bool adjoint(Solver<double>& S, const std::vector<State<double>>& hist, int N,
             std::vector<double>& gout, bool paper = false, const double* lam_term = nullptr,
             double* lam0_out = nullptr) {
    const orc_problem& p = S.p;
    const Grid& g = S.g;
    const Lattice& L = S.L;
    const int Q = L.Q, d = p.dim;
    long dn = (long)S.kref.size();
    gout.assign(dn, 0.0);
    std::vector<double> kp(dn);
    for (long k = 0; k < dn; ++k) kp[k] = kappa_ref_prime(p, S.gamma[k]);
    double h = 1.0 / (double)(p.win_end - p.win_begin + 1);

    State<double> lam, nl;
    lam.resize(g.nodes);
    if (lam_term)   // adjoint of a terminal term <lam_term, s^N>: lambda^N starts there
        for (long m = 0; m < g.nodes; ++m) {
            lam.rho[m] = lam_term[m];
            for (int a = 0; a < 3; ++a) lam.u[a][m] = lam_term[(1 + a) * g.nodes + m];
        }
    std::vector<double> mr(g.nodes), mu[3], e(g.nodes), St((size_t)6 * g.nodes), tmp;
    for (int a = 0; a < 3; ++a) mu[a].assign(g.nodes, 0.0);
    std::vector<double> kappa;
    std::vector<double> us[3];
    const int sidx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    std::vector<double> U3[3], src[3];   // printed variant: 3 U~ of the last moments, J source
    for (int a = 0; a < 3; ++a) {
        U3[a].assign(g.nodes, 0.0);
        src[a].assign(g.nodes, 0.0);
    }

    for (int n = N; n >= 1; --n) {
        const State<double>& sn = hist[n];
        const State<double>& sp = hist[n - 1];
        // (i) direct objective term at level n
        for (int a = 0; a < 3; ++a) std::fill(src[a].begin(), src[a].end(), 0.0);
        if (n >= p.win_begin && n <= p.win_end) {
            for (int z = 0; z < g.n[2]; ++z)
                for (int y = 0; y < g.n[1]; ++y)
                    for (int x = 0; x < g.n[0]; ++x) {
                        if (!in_target(p, x, y, z)) continue;
                        long m = g.idx(x, y, z);
                        if (p.obj_kind == 0) lam.rho[m] += -h / (3.0 * (double)S.count);
                        else
                            for (int a = 0; a < 3; ++a) {
                                lam.u[a][m] += -h * p.obj_dir[a] / (double)S.count;
                                src[a][m] = -h * p.obj_dir[a] / (double)S.count;
                            }
                    }
        }
        // (ii) transpose of the boundary conditions
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    int xa[3] = {x, y, z};
                    if (!on_boundary(g, xa)) continue;
                    int f = winning_face(p, g, xa);
                    int sx[3];
                    inward(g, xa, sx);
                    long b = g.idx(x, y, z), so = g.idx(sx[0], sx[1], sx[2]);
                    int t = p.bc[f];
                    if (t == BC_WALL || t == BC_INLET) {
                        lam.rho[so] += lam.rho[b];
                    } else {
                        int na = f / 2;
                        lam.u[na][so] += lam.u[na][b];
                    }
                    lam.rho[b] = 0.0;
                    for (int a = 0; a < 3; ++a) lam.u[a][b] = 0.0;
                }
        // (iii) transpose of the Brinkman update; e = dJ/dkappa(x, t_n)
        const double* mrow = S.motion + 8 * (long)n;
        if (!transfer<double>(p, g, S.kref, mrow, kappa, us)) return false;
        for (long m = 0; m < g.nodes; ++m) {
            mr[m] = lam.rho[m];
            double ee = 0.0;
            const double kt = kappa[m] + (S.ks.empty() ? 0.0 : S.ks[m]);
            for (int a = 0; a < 3; ++a) {
                if (paper)  // only 3 U~ and the source are divided (Eq. au_ex as printed)
                    mu[a][m] = lam.u[a][m] - (U3[a][m] + src[a][m]) * kt / (1.0 + kt);
                else
                    mu[a][m] = lam.u[a][m] / (1.0 + kt);
                ee += mu[a][m] * (us[a][m] - sn.u[a][m]);
            }
            e[m] = ee;  // boundary nodes carry lam = 0 here, so mu = e = 0 there
        }
        // (iv) design sensitivity through the transposed transfer
        if (p.lx > 0) {
            transfer_T(p, g, mrow, e, tmp);
            for (long k = 0; k < dn; ++k) gout[k] += kp[k] * tmp[k];
        }
        // (v)-(vi) transpose of the gather and of f^eq's dependence on rho and u
        nl.resize(g.nodes);
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    long m = g.idx(x, y, z);
                    double R = 0.0, U[3] = {0, 0, 0}, Sm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                    for (int i = 0; i < Q; ++i) {
                        int xt[3] = {x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]};
                        bool inside = true;
                        for (int a = 0; a < 3; ++a) {
                            if (g.periodic[a]) xt[a] = wrap(xt[a], g.n[a]);
                            else if (xt[a] < 0 || xt[a] >= g.n[a]) inside = false;
                        }
                        if (!inside || on_boundary(g, xt)) continue;
                        long mt = g.idx(xt[0], xt[1], xt[2]);
                        double Ft = mr[mt];
                        for (int a = 0; a < d; ++a) Ft += (double)L.c[i][a] * mu[a][mt];
                        double wF = L.w[i] * Ft;
                        R += wF;
                        for (int a = 0; a < d; ++a) U[a] += (double)L.c[i][a] * wF;
                        for (int al = 0; al < d; ++al)
                            for (int be = 0; be < d; ++be)
                                Sm[al][be] += (double)(L.c[i][al] * L.c[i][be]) * wF;
                    }
                    nl.rho[m] = R;
                    for (int a = 0; a < 3; ++a) U3[a][m] = (a < d) ? 3.0 * U[a] : 0.0;
                    for (int al = 0; al < 3; ++al) {
                        double v = 0.0;
                        if (al < d) {
                            v = 3.0 * U[al] - 3.0 * R * sp.u[al][m];
                            for (int be = 0; be < d; ++be) v += 9.0 * Sm[al][be] * sp.u[be][m];
                        }
                        nl.u[al][m] = v;
                    }
                    for (int al = 0; al < 3; ++al)
                        for (int be = al; be < 3; ++be) St[(size_t)sidx[al][be] * g.nodes + m] = Sm[al][be];
                }
        // (vii) transpose of the gradient: f^eq depends on D_beta u_alpha through
        // A (S_ab + S_ba) c_a c_b, so dJ/d(D_beta u_alpha)(y) = 2 A s~_ab(y); scatter it back
        // through each tap of the derivative operator.
        for (int z = 0; z < g.n[2]; ++z)
            for (int y = 0; y < g.n[1]; ++y)
                for (int x = 0; x < g.n[0]; ++x) {
                    int xa[3] = {x, y, z};
                    long m = g.idx(x, y, z);
                    for (int be = 0; be < d; ++be) {
                        int off[3];
                        double coef[3];
                        int nt = deriv_taps(g, be, xa[be], off, coef);
                        for (int t = 0; t < nt; ++t) {
                            int xb[3] = {x, y, z};
                            xb[be] = wrap(xa[be] + off[t], g.n[be]);
                            long mb = g.idx(xb[0], xb[1], xb[2]);
                            for (int al = 0; al < d; ++al)
                                nl.u[al][mb] +=
                                    coef[t] * 2.0 * p.A * St[(size_t)sidx[al][be] * g.nodes + m];
                        }
                    }
                }
        std::swap(lam, nl);
    }
    if (lam0_out)
        for (long m = 0; m < g.nodes; ++m) {
            lam0_out[m] = lam.rho[m];
            for (int a = 0; a < 3; ++a) lam0_out[(1 + a) * g.nodes + m] = lam.u[a][m];
        }
    return true;
}

template <class T>
void copy_state_out(const Grid& g, const State<T>& s, double* out);

template <>
void copy_state_out<double>(const Grid& g, const State<double>& s, double* out) {
    for (long n = 0; n < g.nodes; ++n) {
        out[n] = s.rho[n];
        for (int a = 0; a < 3; ++a) out[(1 + a) * g.nodes + n] = s.u[a][n];
    }
}

}  // namespace

extern "C" {

const char* orc_error(void) { return g_err.c_str(); }

/* kstatic (may be NULL): static Brinkman coefficient per analysis node (solid velocity 0).
 * lam_term (may be NULL): planes (rho, ux, uy, uz) of a terminal term <lam_term, s^N> added
 * to J; the adjoint then starts from lambda^N = lam_term (a warm-started adjoint). */
static void set_static(Solver<double>& S, const double* kstatic) {
    if (kstatic) S.ks.assign(kstatic, kstatic + S.g.nodes);
}

/* Forward run (Alg. 1): returns J; optionally the final state as planes (rho, ux, uy, uz). */
int orc_forward(const orc_problem* p, const double* gamma, const double* motion, int n_steps,
                const double* init_state, const double* kstatic, const double* lam_term,
                double* J_out, double* final_state) {
    g_err.clear();
    Solver<double> S;
    if (!S.init(*p, gamma, motion)) return 1;
    set_kref_real(S);
    set_static(S, kstatic);
    double J;
    State<double> fin;
    if (!S.forward(n_steps, init_state, J, nullptr, fin, lam_term)) return 1;
    if (J_out) *J_out = J;
    if (final_state) copy_state_out(S.g, fin, final_state);
    return 0;
}

/* Forward run keeping every level, then the exact discrete adjoint: J and dJ/dgamma, and
 * optionally lambda^0 (planes) at the end of the sweep. */
int orc_gradient(const orc_problem* p, const double* gamma, const double* motion, int n_steps,
                 const double* init_state, const double* kstatic, const double* lam_term,
                 double* J_out, double* g_out, double* lam0_out) {
    g_err.clear();
    Solver<double> S;
    if (!S.init(*p, gamma, motion)) return 1;
    set_kref_real(S);
    set_static(S, kstatic);
    double J;
    State<double> fin;
    std::vector<State<double>> hist;
    if (!S.forward(n_steps, init_state, J, &hist, fin, lam_term)) return 1;
    std::vector<double> g;
    if (!adjoint(S, hist, n_steps, g, false, lam_term, lam0_out)) return 1;
    if (J_out) *J_out = J;
    if (g_out) std::memcpy(g_out, g.data(), g.size() * sizeof(double));
    return 0;
}

/* The adjoint of Sec. 2.4 as printed (see adjoint()): J and its dJ/dgamma. */
int orc_gradient_printed(const orc_problem* p, const double* gamma, const double* motion,
                         int n_steps, double* J_out, double* g_out) {
    g_err.clear();
    Solver<double> S;
    if (!S.init(*p, gamma, motion)) return 1;
    set_kref_real(S);
    double J;
    State<double> fin;
    std::vector<State<double>> hist;
    if (!S.forward(n_steps, nullptr, J, &hist, fin)) return 1;
    std::vector<double> g;
    if (!adjoint(S, hist, n_steps, g, true)) return 1;
    if (J_out) *J_out = J;
    if (g_out) std::memcpy(g_out, g.data(), g.size() * sizeof(double));
    return 0;
}

/* Complex-step directional derivative: dJ = Im J(gamma + i h dir) / h, and Re J. */
int orc_complex_step(const orc_problem* p, const double* gamma, const double* motion,
                     int n_steps, const double* kstatic, const double* lam_term,
                     const double* dir, double h, double* dJ_out, double* J_out) {
    g_err.clear();
    Solver<cplx> S;
    if (!S.init(*p, gamma, motion)) return 1;
    S.set_kref_complex(dir, h);
    if (kstatic) S.ks.assign(kstatic, kstatic + S.g.nodes);
    cplx J;
    State<cplx> fin;
    if (!S.forward(n_steps, nullptr, J, nullptr, fin, lam_term)) return 1;
    if (dJ_out) *dJ_out = J.imag() / h;
    if (J_out) *J_out = J.real();
    return 0;
}

/* The transfer alone at one motion row: kappa (nodes) and u_S (3 planes). */
int orc_transfer(const orc_problem* p, const double* gamma, const double* motion_row,
                 double* kappa_out, double* us_out) {
    g_err.clear();
    Solver<double> S;
    if (!S.init(*p, gamma, motion_row)) return 1;
    set_kref_real(S);
    std::vector<double> kappa, us[3];
    if (!transfer<double>(S.p, S.g, S.kref, motion_row, kappa, us)) return 1;
    for (long n = 0; n < S.g.nodes; ++n) {
        kappa_out[n] = kappa[n];
        for (int a = 0; a < 3; ++a) us_out[a * S.g.nodes + n] = us[a][n];
    }
    return 0;
}

/* Transposed transfer of a field e: out(xi) = sum_x W(x - x_ref(xi)) e(x). */
int orc_transfer_T(const orc_problem* p, const double* motion_row, const double* e,
                   double* out) {
    g_err.clear();
    Grid g = make_grid(*p);
    std::vector<double> ev(e, e + g.nodes), o;
    transfer_T(*p, g, motion_row, ev, o);
    std::memcpy(out, o.data(), o.size() * sizeof(double));
    return 0;
}

}  // extern "C"
