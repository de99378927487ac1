/*
 * orca_oracle.c -- plain, slow FP64 CPU oracle of one synchronous ORCA step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  The CUDA
 * library never calls it and shares no code, header or table with it.
 *
 * What one step computes (paper Sec. 3 and 3.1):
 *   - each agent observes radius, position and velocity of nearby agents
 *     (Sec. 3, overview paragraph; the uniform-grid messaging of Sec. 1 is
 *     replaced here by brute force over all agents, which is its definition);
 *   - one half-plane ORCA_{A|B} per neighbour, placed at v_opt + f_{A|B} u
 *     (Sec. 3.1, Fig. 1c); u and the half-plane normal follow the published
 *     ORCA velocity-obstacle geometry;
 *   - the admissible velocity closest to the preferred one (Sec. 3, LP
 *     paragraphs), and when no velocity is admissible, the one of least
 *     penetration (Sec. 3, infeasible paragraph);
 *   - all agents then move with their new velocities in lock step.
 *
 * Discrete decisions (cell of an agent, neighbour candidate test and order,
 * overlap predicate, waypoint advance) are evaluated in IEEE FP32 with the
 * operation order written below, because both implementations must take the
 * same decisions bit for bit.  Everything continuous is FP64.
 *
 * Readings where the paper is silent:
 *   - neighbours: the k nearest candidates with d^2 < R_n^2, ordered by
 *     (d^2, index);
 *   - overlapping pairs use the cut-off-circle construction with tau
 *     replaced by dt (separate within one step);
 *   - left/right leg: det(q, w_rel) > 0 evaluated in FP64 from the FP64
 *     differences, ties go to the right leg;
 *   - the 2D LP result is the Euclidean projection of v_pref onto the
 *     intersection of half-planes and the max-speed disc (unique);
 *   - when that set is empty, t* = min over the disc of the largest signed
 *     penetration, and the result is the projection of v_pref onto the set
 *     of minimisers, i.e. onto the lines relaxed by t*.
 *
 * The LP is solved by enumerating the candidate faces of a projection onto a
 * convex polygon cut by a disc (KKT: the minimiser is v_pref itself, a point
 * on one boundary, or a vertex of two boundaries), which is the plain
 * definition of the problem rather than an incremental algorithm.
 *
 * Every function here is pinned by the test suite to closed forms, brute
 * force or invariants.  Parity unpinned: how closely an FP32 implementation
 * must agree with this oracle at ill-conditioned least-penetration vertices
 * (nearly parallel or nearly tangent planes, where rounding of the line data
 * already moves the answer) has no anchor outside this oracle; the active-set
 * condition number computed here (pinned) marks those agents.
 *
 * Build: cc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared
 * (no fast-math: the FP32 decisions need IEEE rounding and no contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double px, py;   /* point P on the line */
    double dx, dy;   /* unit direction d; admissible side is left of d */
} oline;

/* ------------------------------------------------------------------------ */
/* FP32 discrete decisions                                                   */
/* ------------------------------------------------------------------------ */

/* Cell along one axis: clamp(floor(fl32(fl32(x - o) * inv)), 0, n - 1). */
static int32_t cell_axis(float x, float o, float inv, int32_t n)
{
    float t = x - o;
    t = t * inv;
    float fl = floorf(t);
    if (!(fl >= 0.0f)) return 0;
    if (fl >= (float)(n - 1)) return n - 1;
    return (int32_t)fl;
}

/* Neighbour key d^2 = fl32(fl32(dx*dx) + fl32(dy*dy)), dx = fl32(xb - xa). */
static float key_d2(float xa, float ya, float xb, float yb)
{
    float dx = xb - xa;
    float dy = yb - ya;
    float sx = dx * dx;
    float sy = dy * dy;
    return sx + sy;
}

/* ------------------------------------------------------------------------ */
/* ORCA half-plane of one ordered pair (Sec. 3.1, Fig. 1)                    */
/* ------------------------------------------------------------------------ */

/*
 * q = p_B - p_A, w_rel = v_A - v_B, rho = r_A + r_B.
 * Not overlapping: the velocity obstacle is the cone from the origin tangent
 * to the disc D(q/tau, rho/tau), truncated by that disc.  u is the vector from
 * w_rel to the closest point of the obstacle's boundary; the half-plane
 * boundary passes through v_A + f u with its admissible side facing away
 * from the obstacle.  Overlapping: the same cut-off construction with tau
 * replaced by dt.
 */
static void pair_line(double pax, double pay, double vax, double vay, double ra,
                      double pbx, double pby, double vbx, double vby, double rb,
                      double f, double tau, double dt, int overlap, oline *L)
{
    double qx = pbx - pax, qy = pby - pay;
    double wrx = vax - vbx, wry = vay - vby;
    double rho = ra + rb;
    double ux, uy, dx, dy;
    if (!overlap) {
        double wx = wrx - qx / tau, wy = wry - qy / tau;
        double wq = wx * qx + wy * qy;
        double ww = wx * wx + wy * wy;
        if (wq < 0.0 && wq * wq > rho * rho * ww) {
            /* closest boundary point is on the cut-off circle */
            double wl = sqrt(ww);
            double hx = wx / wl, hy = wy / wl;
            dx = hy;
            dy = -hx;
            double s = rho / tau - wl;
            ux = s * hx;
            uy = s * hy;
        } else {
            /* closest boundary point is on one of the two legs */
            double qq = qx * qx + qy * qy;
            double l2 = qq - rho * rho;
            double l = l2 > 0.0 ? sqrt(l2) : 0.0;
            double side = qx * wry - qy * wrx;   /* det(q, w_rel) */
            if (side > 0.0) {
                dx = (qx * l - qy * rho) / qq;
                dy = (qx * rho + qy * l) / qq;
            } else {
                dx = -(qx * l + qy * rho) / qq;
                dy = -(-qx * rho + qy * l) / qq;
            }
            double proj = wrx * dx + wry * dy;
            ux = proj * dx - wrx;
            uy = proj * dy - wry;
        }
    } else {
        double wx = wrx - qx / dt, wy = wry - qy / dt;
        double wl = sqrt(wx * wx + wy * wy);
        double hx, hy;
        if (wl > 0.0) {
            hx = wx / wl;
            hy = wy / wl;
        } else {
            /* degenerate: relative velocity exactly q/dt; push apart along -q,
               or along -x for coincident agents */
            double ql = sqrt(qx * qx + qy * qy);
            if (ql > 0.0) { hx = -qx / ql; hy = -qy / ql; }
            else { hx = -1.0; hy = 0.0; }
        }
        dx = hy;
        dy = -hx;
        double s = rho / dt - wl;
        ux = s * hx;
        uy = s * hy;
    }
    L->px = vax + f * ux;
    L->py = vay + f * uy;
    L->dx = dx;
    L->dy = dy;
}

/* ------------------------------------------------------------------------ */
/* LP: projection onto half-planes relaxed by t, intersected with a disc     */
/* ------------------------------------------------------------------------ */

/* penetration of v into line i: det(d, P - v) = c - n.v, n = (-dy, dx) */
static double pen(const oline *L, double vx, double vy)
{
    return L->dx * (L->py - vy) - L->dy * (L->px - vx);
}

static int feasible(const oline *L, int n, double t, double vmax,
                    double vx, double vy, double slack)
{
    double r2 = vx * vx + vy * vy;
    double lim = vmax * (1.0 + slack) + slack;
    if (r2 > lim * lim) return 0;
    for (int i = 0; i < n; ++i) {
        double c = L[i].dx * L[i].py - L[i].dy * L[i].px;
        double tol = slack * (1.0 + vmax + fabs(c) + fabs(t));
        if (pen(&L[i], vx, vy) - t > tol) return 0;
    }
    return 1;
}

typedef struct {
    double bx, by, bd;
    int have;
} best_t;

static void consider(best_t *b, const oline *L, int n, double t, double vmax,
                     double vpx, double vpy, double vx, double vy, double slack)
{
    if (!(vx == vx) || !(vy == vy)) return;
    if (!feasible(L, n, t, vmax, vx, vy, slack)) return;
    double ex = vx - vpx, ey = vy - vpy;
    double d = ex * ex + ey * ey;
    if (!b->have || d < b->bd) {
        b->have = 1;
        b->bd = d;
        b->bx = vx;
        b->by = vy;
    }
}

/*
 * Projection of vp onto {v : det(d_i, P_i - v) <= t for all i} and |v| <= vmax
 * by enumeration of every candidate face.  Returns 1 and writes the point if
 * a feasible candidate exists.
 */
static int project_enum(const oline *L, int n, double t, double vmax,
                        double vpx, double vpy, double slack,
                        double *ox, double *oy)
{
    best_t b = {0.0, 0.0, 0.0, 0};
    double r2 = vmax * vmax;
    consider(&b, L, n, t, vmax, vpx, vpy, vpx, vpy, slack);
    double vl = sqrt(vpx * vpx + vpy * vpy);
    if (vl > 0.0)
        consider(&b, L, n, t, vmax, vpx, vpy, vmax * vpx / vl, vmax * vpy / vl, slack);
    for (int i = 0; i < n; ++i) {
        double nix = -L[i].dy, niy = L[i].dx;
        double bi = (L[i].dx * L[i].py - L[i].dy * L[i].px) - t; /* n_i.v = b_i */
        /* projection onto the line */
        double s = bi - (nix * vpx + niy * vpy);
        consider(&b, L, n, t, vmax, vpx, vpy, vpx + s * nix, vpy + s * niy, slack);
        /* line meets the circle; a line tangent to it (up to rounding)
           meets it only at the tangent point, which is the single minimiser
           when one half-plane alone attains t* on the circle */
        double h2 = r2 - bi * bi;
        if (h2 >= 0.0) {
            double h = sqrt(h2);
            double cx = bi * nix, cy = bi * niy;
            consider(&b, L, n, t, vmax, vpx, vpy, cx + h * L[i].dx, cy + h * L[i].dy, slack);
            consider(&b, L, n, t, vmax, vpx, vpy, cx - h * L[i].dx, cy - h * L[i].dy, slack);
        } else {
            double sg = bi > 0.0 ? vmax : -vmax;
            consider(&b, L, n, t, vmax, vpx, vpy, sg * nix, sg * niy, slack);
        }
        /* line meets another line */
        for (int j = i + 1; j < n; ++j) {
            double njx = -L[j].dy, njy = L[j].dx;
            double bj = (L[j].dx * L[j].py - L[j].dy * L[j].px) - t;
            double det = nix * njy - niy * njx;
            if (fabs(det) <= 1e-14) continue;
            double x = (bi * njy - bj * niy) / det;
            double y = (nix * bj - njx * bi) / det;
            consider(&b, L, n, t, vmax, vpx, vpy, x, y, slack);
        }
    }
    if (!b.have) return 0;
    *ox = b.bx;
    *oy = b.by;
    return 1;
}

static double gmax(const oline *L, int n, double vx, double vy)
{
    double g = -INFINITY;
    for (int i = 0; i < n; ++i) {
        double p = pen(&L[i], vx, vy);
        if (p > g) g = p;
    }
    return g;
}

/*
 * t* = min over |v| <= vmax of max_i det(d_i, P_i - v) (least penetration,
 * Sec. 3).  The minimum of a convex piecewise-linear function over a disc is
 * attained at a vertex of three planes, at a point of the circle where two
 * planes are equal, or at the point of the circle that minimises one plane;
 * every such candidate is evaluated.  Returns -inf for no lines.
 */
static double tstar_enum(const oline *L, int n, double vmax, double *ax, double *ay)
{
    double best = INFINITY, bx = 0.0, by = 0.0;
    double lim = vmax * (1.0 + 1e-12);
    if (n == 0) {
        *ax = 0.0;
        *ay = 0.0;
        return -INFINITY;
    }
#define TRY(X, Y)                                                   \
    do {                                                            \
        double _x = (X), _y = (Y);                                  \
        if (_x * _x + _y * _y <= lim * lim) {                       \
            double _g = gmax(L, n, _x, _y);                         \
            if (_g < best) { best = _g; bx = _x; by = _y; }         \
        }                                                           \
    } while (0)
    for (int i = 0; i < n; ++i) {
        double nix = -L[i].dy, niy = L[i].dx;
        double ci = L[i].dx * L[i].py - L[i].dy * L[i].px;
        TRY(vmax * nix, vmax * niy);
        for (int j = i + 1; j < n; ++j) {
            double njx = -L[j].dy, njy = L[j].dx;
            double cj = L[j].dx * L[j].py - L[j].dy * L[j].px;
            /* equal penetration of i and j: (n_j - n_i).v = c_j - c_i */
            double ax_ = njx - nix, ay_ = njy - niy;
            double bb = cj - ci;
            double aa = ax_ * ax_ + ay_ * ay_;
            if (aa > 1e-20) {
                double x0 = ax_ * bb / aa, y0 = ay_ * bb / aa;
                double h2 = vmax * vmax - (x0 * x0 + y0 * y0);
                if (h2 >= 0.0) {
                    double h = sqrt(h2 / aa);
                    TRY(x0 - h * ay_, y0 + h * ax_);
                    TRY(x0 + h * ay_, y0 - h * ax_);
                }
            }
            for (int l = j + 1; l < n; ++l) {
                double nlx = -L[l].dy, nly = L[l].dx;
                double cl = L[l].dx * L[l].py - L[l].dy * L[l].px;
                double a2x = nlx - nix, a2y = nly - niy;
                double b2 = cl - ci;
                double det = ax_ * a2y - ay_ * a2x;
                if (fabs(det) <= 1e-14) continue;
                TRY((bb * a2y - b2 * ay_) / det, (ax_ * b2 - a2x * bb) / det);
            }
        }
    }
#undef TRY
    *ax = bx;
    *ay = by;
    return best;
}

/* Active boundaries at v and the conditioning of the best-conditioned pair
   of them (1 / sin of the angle between the two boundaries). */
static double active_cond(const oline *L, int n, double t, double vmax,
                          double vx, double vy, uint32_t *mask, int *on_circle)
{
    double scale = 1.0 + vmax;
    uint32_t m = 0;
    int nact = 0;
    int idx[64];
    for (int i = 0; i < n; ++i) {
        double c = L[i].dx * L[i].py - L[i].dy * L[i].px;
        if (fabs(pen(&L[i], vx, vy) - t) <= 1e-9 * (scale + fabs(c) + fabs(t))) {
            if (i < 32) m |= (1u << i);
            if (nact < 64) idx[nact++] = i;
        }
    }
    double vl = sqrt(vx * vx + vy * vy);
    int circ = fabs(vl - vmax) <= 1e-9 * scale;
    *mask = m;
    *on_circle = circ;
    double best = INFINITY;
    for (int a = 0; a < nact; ++a) {
        for (int b = a + 1; b < nact; ++b) {
            double s = fabs(L[idx[a]].dx * L[idx[b]].dy - L[idx[a]].dy * L[idx[b]].dx);
            if (s > 0.0 && 1.0 / s < best) best = 1.0 / s;
        }
        if (circ && vl > 0.0) {
            double s = fabs(L[idx[a]].dx * vx + L[idx[a]].dy * vy) / vl;
            if (s > 0.0 && 1.0 / s < best) best = 1.0 / s;
        }
    }
    if (nact + circ < 2) return 1.0;
    return best;
}

/*
 * Whether two half-planes that attain t* at the minimiser (ax, ay) point in
 * exactly opposite directions.  Only then is the set of least-penetration
 * velocities a segment (a valley between the two); otherwise the maximum of
 * the penetrations grows in every direction and the minimiser is the point.
 */
static int valley_at(const oline *L, int n, double t, double vmax, double ax, double ay)
{
    double scale = 1.0 + vmax;
    for (int i = 0; i < n; ++i) {
        double ci = L[i].dx * L[i].py - L[i].dy * L[i].px;
        if (fabs(pen(&L[i], ax, ay) - t) > 1e-9 * (scale + fabs(ci) + fabs(t))) continue;
        for (int j = i + 1; j < n; ++j) {
            double cj = L[j].dx * L[j].py - L[j].dy * L[j].px;
            if (fabs(pen(&L[j], ax, ay) - t) > 1e-9 * (scale + fabs(cj) + fabs(t))) continue;
            double dot = L[i].dx * L[j].dx + L[i].dy * L[j].dy;
            double det = L[i].dx * L[j].dy - L[i].dy * L[j].dx;
            if (dot < 0.0 && fabs(det) <= 1e-12) return 1;
        }
    }
    return 0;
}

/*
 * The velocity LP of one agent.  Writes v*, t* and returns flags:
 *   bit0 = constraints infeasible (t* > 0, least-penetration result)
 *   bit1 = enumeration found no candidate even with widened tolerances
 *   bit3 = result on the max-speed circle
 */
static int lp_solve(const oline *L, int n, double vmax, double vpx, double vpy,
                    double *ox, double *oy, double *otstar, double *ocond,
                    uint32_t *omask)
{
    int flags = 0;
    double ax, ay;
    double ts = tstar_enum(L, n, vmax, &ax, &ay);
    double t = ts > 0.0 ? ts : 0.0;
    if (ts > 0.0) flags |= 1;
    double slack = 1e-11;
    int ok = 0;
    if (ts > 0.0 && !valley_at(L, n, ts, vmax, ax, ay)) {
        /* a single least-penetration velocity: the enumerated vertex itself
           (projecting onto the relaxed set would only approximate it) */
        *ox = ax;
        *oy = ay;
        ok = 1;
    }
    for (int tries = 0; tries < 4 && !ok; ++tries, slack *= 100.0)
        ok = project_enum(L, n, t, vmax, vpx, vpy, slack, ox, oy);
    if (!ok) {
        flags |= 2;
        *ox = ax;
        *oy = ay;
    }
    *otstar = ts;
    int circ = 0;
    uint32_t mask = 0;
    double cond = active_cond(L, n, t, vmax, *ox, *oy, &mask, &circ);
    if (circ) flags |= 8;
    if (ocond) *ocond = cond;
    if (omask) *omask = mask;
    return flags;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Cell id cy*nx + cx of each agent (FP32 decision, paper Sec. 1 grid).  The
   paper fixes no cell shape; cells are w x h rectangles, inv_cell_x =
   fl32(1/w) along x and inv_cell_y = fl32(1/h) along y (square when equal). */
void oracle_cells(int n, const float *px, const float *py, float ox, float oy,
                  float inv_cell_x, float inv_cell_y, int nx, int ny, int32_t *out)
{
    for (int i = 0; i < n; ++i) {
        int32_t cx = cell_axis(px[i], ox, inv_cell_x, nx);
        int32_t cy = cell_axis(py[i], oy, inv_cell_y, ny);
        out[i] = cy * nx + cx;
    }
}

/* ORCA half-plane of one ordered pair, out = {P_x, P_y, d_x, d_y}. */
void oracle_pair_line(double pax, double pay, double vax, double vay, double ra,
                      double pbx, double pby, double vbx, double vby, double rb,
                      double f, double tau, double dt, int overlap, double *out)
{
    oline L;
    pair_line(pax, pay, vax, vay, ra, pbx, pby, vbx, vby, rb, f, tau, dt, overlap, &L);
    out[0] = L.px;
    out[1] = L.py;
    out[2] = L.dx;
    out[3] = L.dy;
}

/* LP of one agent from explicit lines (4 doubles each: P_x, P_y, d_x, d_y).
   out = {v_x, v_y, t*, cond}; returns the flags of lp_solve. */
int oracle_lp(int n, const double *lines, double vmax, double vpx, double vpy,
              double *out, uint32_t *mask)
{
    oline L[64];
    if (n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        L[i].px = lines[4 * i + 0];
        L[i].py = lines[4 * i + 1];
        L[i].dx = lines[4 * i + 2];
        L[i].dy = lines[4 * i + 3];
    }
    return lp_solve(L, n, vmax, vpx, vpy, &out[0], &out[1], &out[2], &out[3], mask);
}

/* Projection of vp onto the lines relaxed by t (and the disc), exported for
   the tests of the tie-break rule.  Returns 0 when the set is empty. */
int oracle_project(int n, const double *lines, double t, double vmax,
                   double vpx, double vpy, double *out)
{
    oline L[64];
    if (n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        L[i].px = lines[4 * i + 0];
        L[i].py = lines[4 * i + 1];
        L[i].dx = lines[4 * i + 2];
        L[i].dy = lines[4 * i + 3];
    }
    return project_enum(L, n, t, vmax, vpx, vpy, 1e-11, &out[0], &out[1]);
}

/*
 * One synchronous ORCA step for the agents listed in sel (all when sel is
 * NULL), reading the step-t state of every agent.
 *
 * State arrays are FP64; the discrete decisions use their FP32 roundings, so
 * an FP32 state passed as FP64 reproduces the FP32 specification exactly.
 * f4 = {f[0][0], f[0][1], f[1][0], f[1][1]} indexed by (type_A, type_B).
 * route/wpx/wpy/wp_idx may be NULL (every agent then follows its goal);
 * dvx/dvy (per-agent preferred-velocity offsets) may be NULL.
 *
 * Per selected agent s (index sel[s]) the outputs are
 *   out_v[2s..], out_p[2s..]         new velocity and position (FP64)
 *   out_wp[s]                        waypoint index after the advance rule
 *   out_nbr[s*k..], out_cnt[s]       neighbour indices in constraint order
 *   out_flags[s]                     lp flags | 4 if any neighbour overlaps
 *   out_tstar[s], out_cond[s]        least penetration t*, active conditioning
 *   out_lines[(s*k + m)*4..]         the constraint lines (may be NULL)
 *   out_mask[s]                      active constraint bitmask (may be NULL)
 * Returns 0, or -1 for invalid arguments.
 */
int oracle_step(int n, const double *px, const double *py, const double *vx,
                const double *vy, const double *gx, const double *gy,
                const double *radius, const double *vmax, const uint8_t *type,
                const int32_t *route, const double *wpx, const double *wpy,
                int n_wp, const uint8_t *wp_idx, const double *dvx,
                const double *dvy, double neighbor_dist, int k, double tau,
                double dt, const double *f4, double turn_rate, double accel,
                int n_sel, const int32_t *sel,
                double *out_v, double *out_p, uint8_t *out_wp, int32_t *out_nbr,
                int32_t *out_cnt, uint8_t *out_flags, double *out_tstar,
                double *out_cond, double *out_lines, uint32_t *out_mask)
{
    if (n < 0 || k < 0 || k > 64 || n_sel < 0) return -1;
    const float R = (float)neighbor_dist;
    const float R2 = R * R;
#pragma omp parallel for schedule(dynamic, 16)
    for (int s = 0; s < n_sel; ++s) {
        int a = sel ? sel[s] : s;
        float xa = (float)px[a], ya = (float)py[a];
        float raf = (float)radius[a];
        /* k nearest candidates by (d^2, index), brute force over all agents */
        float bd[64];
        int32_t bi[64];
        int cnt = 0;
        for (int b = 0; b < n && k > 0; ++b) {
            if (b == a) continue;
            float d2 = key_d2(xa, ya, (float)px[b], (float)py[b]);
            if (!(d2 < R2)) continue;
            if (cnt == k && !(d2 < bd[k - 1] || (d2 == bd[k - 1] && b < bi[k - 1])))
                continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && (d2 < bd[pos - 1] || (d2 == bd[pos - 1] && b < bi[pos - 1]))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = d2;
            bi[pos] = b;
            if (cnt < k) ++cnt;
        }
        /* preferred velocity toward the goal or the current waypoint */
        double tx = gx[a], ty = gy[a];
        int wi = 0;
        if (route && route[a] >= 0) {
            wi = wp_idx[a];
            int base = route[a] * n_wp;
            float wdx = (float)wpx[base + wi] - (float)px[a];
            float wdy = (float)wpy[base + wi] - (float)py[a];
            float w2 = wdx * wdx + wdy * wdy;
            float rr = raf * raf;
            if (wi < n_wp - 1 && w2 <= rr) ++wi;
            tx = wpx[base + wi];
            ty = wpy[base + wi];
        }
        double gpx = tx - px[a], gpy = ty - py[a];
        double gl = sqrt(gpx * gpx + gpy * gpy);
        double vpx = 0.0, vpy = 0.0;
        if (gl > 0.0) {
            double sc = vmax[a] / gl;
            if (sc > 1.0 / dt) sc = 1.0 / dt;
            vpx = gpx * sc;
            vpy = gpy * sc;
        }
        if (dvx) {
            vpx += dvx[a];
            vpy += dvy[a];
        }
        /* one ORCA line per neighbour */
        oline L[64 + 3];   /* k ORCA lines + up to 3 kinematic ones */
        int any_overlap = 0;
        for (int m = 0; m < cnt; ++m) {
            int b = bi[m];
            float rbf = (float)radius[b];
            float rs = raf + rbf;
            float rr = rs * rs;
            int overlap = bd[m] <= rr;
            any_overlap |= overlap;
            double f = f4[type[a] * 2 + type[b]];
            pair_line(px[a], py[a], vx[a], vy[a], radius[a], px[b], py[b], vx[b],
                      vy[b], radius[b], f, tau, dt, overlap, &L[m]);
        }
        /* vehicles' kinematic half-planes (the paper's proposed extension,
           Sec. 5), after the ORCA ones: for a moving vehicle (|v| >= 0.1 m/s,
           an FP32 decision) the new heading stays within +-turn_rate*dt of the
           current one (two half-planes through the origin), and the forward
           speed grows by at most accel*dt (v . h <= |v| + accel dt); a slower
           vehicle gets only the latter, along its preferred velocity */
        int nl = cnt;
        if (type[a] != 0 && (turn_rate > 0.0 || accel > 0.0)) {
            float fvx = (float)vx[a], fvy = (float)vy[a];
            float sx = fvx * fvx, sy = fvy * fvy;
            float sp2f = sx + sy;
            int moving = sp2f >= 0.01f;
            double hx = 0.0, hy = 0.0, sp = 0.0;
            if (moving) {
                sp = sqrt(vx[a] * vx[a] + vy[a] * vy[a]);
                hx = vx[a] / sp;
                hy = vy[a] / sp;
            } else {
                double pl = sqrt(vpx * vpx + vpy * vpy);
                if (pl > 0.0) { hx = vpx / pl; hy = vpy / pl; }
            }
            if (moving && turn_rate > 0.0) {
                double th = turn_rate * dt, c = cos(th), sn = sin(th);
                /* left ray R(+th) h: admissible to its right, d = -R(+th) h */
                L[nl].px = 0.0; L[nl].py = 0.0;
                L[nl].dx = -(c * hx - sn * hy); L[nl].dy = -(sn * hx + c * hy);
                ++nl;
                /* right ray R(-th) h: admissible to its left */
                L[nl].px = 0.0; L[nl].py = 0.0;
                L[nl].dx = c * hx + sn * hy; L[nl].dy = -sn * hx + c * hy;
                ++nl;
            }
            if (accel > 0.0 && (hx != 0.0 || hy != 0.0)) {
                double smax = sp + accel * dt;
                L[nl].px = smax * hx; L[nl].py = smax * hy;
                L[nl].dx = -hy; L[nl].dy = hx;
                ++nl;
            }
        }
        double nvx, nvy, ts, cond;
        uint32_t mask;
        int fl = lp_solve(L, nl, vmax[a], vpx, vpy, &nvx, &nvy, &ts, &cond, &mask);
        if (any_overlap) fl |= 4;
        out_v[2 * s] = nvx;
        out_v[2 * s + 1] = nvy;
        out_p[2 * s] = px[a] + dt * nvx;
        out_p[2 * s + 1] = py[a] + dt * nvy;
        if (out_wp) out_wp[s] = (uint8_t)wi;
        if (out_nbr) {
            for (int m = 0; m < k; ++m) out_nbr[(size_t)s * k + m] = m < cnt ? bi[m] : -1;
        }
        if (out_cnt) out_cnt[s] = cnt;
        if (out_flags) out_flags[s] = (uint8_t)fl;
        if (out_tstar) out_tstar[s] = ts;
        if (out_cond) out_cond[s] = cond;
        if (out_mask) out_mask[s] = mask;
        if (out_lines) {
            for (int m = 0; m < k; ++m) {
                double *o = out_lines + ((size_t)s * k + m) * 4;
                if (m < cnt) {
                    o[0] = L[m].px; o[1] = L[m].py; o[2] = L[m].dx; o[3] = L[m].dy;
                } else {
                    o[0] = o[1] = o[2] = o[3] = 0.0;
                }
            }
        }
    }
    return 0;
}
