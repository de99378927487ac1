// orca_math.cuh -- per-agent device math of the ORCA step (FP32).
//
// Discrete decisions (cell, neighbour key, overlap, waypoint advance, leg
// side) use explicitly rounded intrinsics in a fixed order so that they
// never get contracted into FMAs: they are part of the specification both
// implementations evaluate identically.  Everything else is plain FP32.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace orca {

// Cell along one axis: clamp(floor(fl32(fl32(x - o) * inv)), 0, n - 1).
__device__ __forceinline__ int cell_axis(float x, float o, float inv, int n) {
    float t = __fmul_rn(__fsub_rn(x, o), inv);
    float fl = floorf(t);
    if (!(fl >= 0.0f)) return 0;
    if (fl >= (float)(n - 1)) return n - 1;
    return (int)fl;
}

// Unsigned key ordered like the float x (negative values reversed, -0 just
// below +0, NaNs at the ends): the order of agents inside a grid cell.
__device__ __forceinline__ uint32_t x_order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Neighbour key d^2 = fl32(fl32(dx*dx) + fl32(dy*dy)), dx = fl32(xb - xa).
__device__ __forceinline__ float key_d2(float xa, float ya, float xb, float yb) {
    float dx = __fsub_rn(xb, xa);
    float dy = __fsub_rn(yb, ya);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Which leg of the velocity obstacle is closer: det(q, w_rel) > 0 means the
// left leg (ties go right).  The decision is defined by the FP64 evaluation
// q = p_B - p_A, w = v_A - v_B, det = q_x w_y - q_y w_x (no contraction).  An
// FP32 filter with a rigorous error bound settles almost every pair; an
// exactly zero w or q (two agents with equal velocities, e.g. both at rest,
// or at one point) gives det = 0, the right leg; only the remaining
// near-zero determinants pay for the FP64 evaluation.
__device__ __forceinline__ bool leg_left(float pax, float pay, float pbx, float pby,
                                         float vax, float vay, float vbx, float vby) {
    float qx = __fsub_rn(pbx, pax), qy = __fsub_rn(pby, pay);
    float wx = __fsub_rn(vax, vbx), wy = __fsub_rn(vay, vby);
    float a = __fmul_rn(qx, wy), b = __fmul_rn(qy, wx);
    float det = __fsub_rn(a, b);
    // |det32 - det_exact| <= ~4u (|a| + |b|); 10u leaves margin
    float bound = 5.97e-7f * (fabsf(a) + fabsf(b));
    if (fabsf(det) > bound) return det > 0.0f;
    // the FP32 difference of two floats is zero only when they are equal,
    // so these are exact zeros of q or w (and of the FP64 determinant)
    if ((wx == 0.0f && wy == 0.0f) || (qx == 0.0f && qy == 0.0f)) return false;
    double qx64 = __dsub_rn((double)pbx, (double)pax);
    double qy64 = __dsub_rn((double)pby, (double)pay);
    double wx64 = __dsub_rn((double)vax, (double)vbx);
    double wy64 = __dsub_rn((double)vay, (double)vby);
    double d64 = __dsub_rn(__dmul_rn(qx64, wy64), __dmul_rn(qy64, wx64));
    return d64 > 0.0;
}

// Squared leg length |q|^2 - rho^2 of the velocity obstacle.  For a pair
// close to touching, the FP32 difference of two nearly equal squares keeps
// only a few correct bits (|q|^2 = 1.000038 against rho^2 = 1 loses three
// digits), and the leg direction inherits that error.  There it is redone
// from error-free FP32 transformations: each square split exactly into a
// rounded product and its FMA residual, the radius sum into its rounded
// value and remainder (two-sum), and |q|^2's leading part taken exactly as
// a two-sum.  The two leading parts, |q|^2 and rho^2, lie within a factor 2
// of each other here, so their difference is exact (Sterbenz), and only the
// residuals, each below one ulp of rho^2, are added with rounding.  The
// result is the exact value up to one final rounding and a few units of
// 2^-47 rho^2 (as accurate as an FP64 evaluation, without the FP64 pipe).
__device__ __forceinline__ float leg_l2(float qx, float qy, float ra, float rb, float qq,
                                        float rho2) {
    float l2 = qq - rho2;
    if (l2 < 0.015625f * qq) {
        // qx^2 = px + ex, qy^2 = py + ey, s^2 = ps + es exactly
        const float px = __fmul_rn(qx, qx), ex = __fmaf_rn(qx, qx, -px);
        const float py = __fmul_rn(qy, qy), ey = __fmaf_rn(qy, qy, -py);
        // ra + rb = s + e exactly
        const float s = __fadd_rn(ra, rb);
        const float sb = __fsub_rn(s, ra);
        const float e = __fadd_rn(__fsub_rn(ra, __fsub_rn(s, sb)), __fsub_rn(rb, sb));
        const float ps = __fmul_rn(s, s), es = __fmaf_rn(s, s, -ps);
        // px + py = S + se exactly
        const float S = __fadd_rn(px, py);
        const float Sb = __fsub_rn(S, px);
        const float se = __fadd_rn(__fsub_rn(px, __fsub_rn(S, Sb)), __fsub_rn(py, Sb));
        // |q|^2 - rho^2 = (S - ps) + (se + ex + ey - es - 2 s e - e^2); e^2 is
        // below 2^-48 rho^2 and left out
        const float hi = __fsub_rn(S, ps);
        const float lo = __fsub_rn(__fsub_rn(__fadd_rn(__fadd_rn(se, ex), ey), es),
                                   __fmul_rn(__fadd_rn(s, s), e));
        l2 = __fadd_rn(hi, lo);
    }
    return l2;
}

// ORCA half-plane of agent A against neighbour B (paper Sec. 3.1, Fig. 1).
// q = p_B - p_A, w_rel = v_A - v_B, rho = r_A + r_B.  The velocity obstacle is
// the cone from the origin tangent to D(q/tau, rho/tau), cut off by that
// disc; u runs from w_rel to its closest boundary point.  Overlapping pairs
// use the cut-off construction with tau replaced by dt.  The line passes
// through v_A + f u; its admissible side is left of the unit direction d.
// Returned as (P_x, P_y, d_x, d_y); cap reports whether a non-overlapping
// pair took the cut-off circle (true) or a leg (false).
__device__ __forceinline__ float4 orca_line(float pax, float pay, float vax, float vay,
                                            float ra, float pbx, float pby, float vbx,
                                            float vby, float rb, float f, float inv_tau,
                                            float inv_dt, bool overlap, bool& cap) {
    cap = false;
    float qx = pbx - pax, qy = pby - pay;
    float wrx = vax - vbx, wry = vay - vby;
    float rho = ra + rb;
    float ux, uy, dx, dy;
    if (!overlap) {
        float wx = wrx - qx * inv_tau, wy = wry - qy * inv_tau;
        float wq = wx * qx + wy * qy;
        float ww = wx * wx + wy * wy;
        float rho2 = rho * rho;
        if (wq < 0.0f && wq * wq > rho2 * ww) {
            // cut-off circle
            cap = true;
            float wl = sqrtf(ww);
            float hx = wx / wl, hy = wy / wl;
            dx = hy;
            dy = -hx;
            float s = rho * inv_tau - wl;
            ux = s * hx;
            uy = s * hy;
        } else {
            // legs
            float qq = qx * qx + qy * qy;
            float l = sqrtf(fmaxf(leg_l2(qx, qy, ra, rb, qq, rho2), 0.0f));
            bool left = leg_left(pax, pay, pbx, pby, vax, vay, vbx, vby);
            float iq = 1.0f / qq;
            if (left) {
                dx = (qx * l - qy * rho) * iq;
                dy = (qx * rho + qy * l) * iq;
            } else {
                dx = -(qx * l + qy * rho) * iq;
                dy = -(qy * l - qx * rho) * iq;
            }
            float pr = wrx * dx + wry * dy;
            ux = pr * dx - wrx;
            uy = pr * dy - wry;
        }
    } else {
        float wx = wrx - qx * inv_dt, wy = wry - qy * inv_dt;
        float wl = sqrtf(wx * wx + wy * wy);
        float hx, hy;
        if (wl > 0.0f) {
            hx = wx / wl;
            hy = wy / wl;
        } else {
            float ql = sqrtf(qx * qx + qy * qy);
            if (ql > 0.0f) {
                hx = -qx / ql;
                hy = -qy / ql;
            } else {
                hx = -1.0f;
                hy = 0.0f;
            }
        }
        dx = hy;
        dy = -hx;
        float s = rho * inv_dt - wl;
        ux = s * hx;
        uy = s * hy;
    }
    return make_float4(vax + f * ux, vay + f * uy, dx, dy);
}

// det(d, P - v): positive = v violates the half-plane
__device__ __forceinline__ float penetration(float4 L, float vx, float vy) {
    return L.z * (L.y - vy) - L.w * (L.x - vx);
}

// ---------------------------------------------------------------------------
// Active set of the velocity LP, packed in 32 bits for the adjoint:
//   bits 0-1   kind: ACT_PROJ   projection of v_pref onto the admissible set
//                    ACT_VERTEX least-penetration vertex (no v_pref term)
//                    ACT_VALLEY projection of v_pref onto a valley mid-line
//   bit 2      the speed circle |v| = vmax is active
//   bits 3-4   number of active lines (0-3)
//   bits 8-12, 16-20, 24-28   constraint indices of active lines a, b, c
//   bits 13/21/29   line a/b/c was built by the cut-off circle construction
//   bits 14/22/30   line a/b/c is an overlapping pair
// The solver fills kind, circle and indices; the solve kernel adds the
// construction bits of the active lines.
// ---------------------------------------------------------------------------
enum : uint32_t { ACT_PROJ = 0u, ACT_VERTEX = 1u, ACT_VALLEY = 2u };

__host__ __device__ __forceinline__ uint32_t act_pack(uint32_t kind, bool circle, int nl, int a,
                                                      int b, int c) {
    return kind | (circle ? 4u : 0u) | ((uint32_t)nl << 3) | ((uint32_t)(a & 31) << 8) |
           ((uint32_t)(b & 31) << 16) | ((uint32_t)(c & 31) << 24);
}
__host__ __device__ __forceinline__ uint32_t act_kind(uint32_t a) { return a & 3u; }
__host__ __device__ __forceinline__ bool act_circle(uint32_t a) { return (a >> 2) & 1u; }
__host__ __device__ __forceinline__ int act_nlines(uint32_t a) { return (int)((a >> 3) & 3u); }
__host__ __device__ __forceinline__ int act_line(uint32_t a, int m) {
    return (int)((a >> (8 + 8 * m)) & 31u);
}
__host__ __device__ __forceinline__ bool act_cap(uint32_t a, int m) {
    return (a >> (13 + 8 * m)) & 1u;
}
__host__ __device__ __forceinline__ bool act_overlap(uint32_t a, int m) {
    return (a >> (14 + 8 * m)) & 1u;
}

// ---------------------------------------------------------------------------
// Velocity LP (paper Sec. 3, LP paragraphs).  Lines live in shared memory at
// L[i * stride].  Interval bounds divide by determinants of unit directions
// (|den| <= 2), so the fast 2-ulp division is safe and costs two
// instructions instead of the IEEE sequence.  The objective is the Euclidean distance to v_pref, so the
// incremental scheme is exact: when the current optimum violates line i, the
// new optimum lies on line i, and a 1D problem on that line with the earlier
// lines and the speed disc finds it.
// ---------------------------------------------------------------------------

// Rounding allowance of the LP's emptiness tests, in m/s.  Intervals whose
// ends cross by less than this are rounding, not infeasibility: half-planes
// of f = 0 pairs all pass through the agent's own velocity, and when that
// lies on the speed circle their exact common point meets the circle's
// rounded end (a vehicle at full speed among pedestrians).
__device__ __forceinline__ float lp_tol(float vmax) { return 1e-5f * (1.0f + vmax); }

// 1D problem on line i: the point of line i closest to v_pref that keeps
// lines 0..i-1 and the disc.  Returns false when that set is empty.
// bound: the constraint that binds the result on line i (-2 none, -1 the
// speed circle, j >= 0 line j).
__device__ __forceinline__ bool lp1_project(const float4* __restrict__ L, int stride, int i,
                                            float vmax, float vpx, float vpy, float& ox,
                                            float& oy, int& work, int& bound) {
    float4 li = L[i * stride];
    const float tol = lp_tol(vmax);
    float dot = li.x * li.z + li.y * li.w;
    float disc = dot * dot + vmax * vmax - (li.x * li.x + li.y * li.y);
    if (disc < -tol * (1.0f + vmax)) return false;
    float sq = sqrtf(fmaxf(disc, 0.0f));
    float tl = -dot - sq, tr = -dot + sq;
    int jl = -1, jr = -1;
    for (int j = 0; j < i; ++j) {
        ++work;
        float4 lj = L[j * stride];
        float den = li.z * lj.w - li.w * lj.z;                     // det(d_i, d_j)
        float num = lj.z * (li.y - lj.y) - lj.w * (li.x - lj.x);   // det(d_j, P_i - P_j)
        if (den == 0.0f) {
            if (num < -tol) return false;
            continue;
        }
        float t = __fdividef(num, den);
        if (den > 0.0f) {
            if (t < tr) jr = j;
            tr = fminf(tr, t);
        } else {
            if (t > tl) jl = j;
            tl = fmaxf(tl, t);
        }
        if (tl > tr + tol) return false;
    }
    float t0 = li.z * (vpx - li.x) + li.w * (vpy - li.y);
    float t = fminf(fmaxf(t0, tl), tr);
    bound = (t0 > tr) ? jr : ((t0 < tl) ? jl : -2);
    ox = li.x + t * li.z;
    oy = li.y + t * li.w;
    return true;
}

// Projection of v_pref onto the half-planes and the disc.  Returns n on
// success, else the index of the line whose 1D problem was empty (v keeps
// the optimum of the lines before it).
__device__ __forceinline__ int lp2_project(const float4* __restrict__ L, int stride, int n,
                                           float vmax, float vpx, float vpy, float& vx,
                                           float& vy, int& work, uint32_t& act) {
    float vp2 = vpx * vpx + vpy * vpy;
    if (vp2 > vmax * vmax) {
        float s = vmax / sqrtf(vp2);
        vx = vpx * s;
        vy = vpy * s;
        act = act_pack(ACT_PROJ, true, 0, 0, 0, 0);
    } else {
        vx = vpx;
        vy = vpy;
        act = act_pack(ACT_PROJ, false, 0, 0, 0, 0);
    }
    for (int i = 0; i < n; ++i) {
        float4 li = L[i * stride];
        if (penetration(li, vx, vy) > 0.0f) {
            float ox, oy;
            int bound;
            if (!lp1_project(L, stride, i, vmax, vpx, vpy, ox, oy, work, bound)) return i;
            vx = ox;
            vy = oy;
            act = bound >= 0 ? act_pack(ACT_PROJ, false, 2, i, bound, 0)
                             : act_pack(ACT_PROJ, bound == -1, 1, i, 0, 0);
        }
    }
    return n;
}

// Boundary of {v : det_j(v) <= det_i(v)} as a line with its admissible side
// on the left.  With n = (-d_y, d_x) and c = det(d, P) = n . P the set is
// (n_j - n_i) . v >= c_j - c_i: normal a = n_j - n_i, offset b = c_j - c_i,
// direction (a_y, -a_x)/|a|, anchored at its closest point to the origin
// a b / |a|^2 (an intersection point would run off to infinity for nearly
// opposite lines and lose all FP32 precision).  Returns false for parallel
// lines of the same direction (one of them dominates everywhere).
__device__ __forceinline__ bool bisector(float4 li, float4 lj, float4& b) {
    const float ax = li.w - lj.w;          // n_j - n_i, n = (-d_y, d_x)
    const float ay = lj.z - li.z;
    const float a2 = ax * ax + ay * ay;
    if (a2 <= 1e-12f) return false;
    const float ci = li.z * li.y - li.w * li.x;
    const float cj = lj.z * lj.y - lj.w * lj.x;
    const float s = __fdividef(cj - ci, a2);
    const float inv = rsqrtf(a2);
    b = make_float4(ax * s, ay * s, ay * inv, -ax * inv);
    return true;
}

// Least penetration (paper Sec. 3, infeasible-set paragraph):
// t* = min over |v| <= vmax of max_i det(d_i, P_i - v), by the incremental
// LP in (v, t): when the optimum violates plane i, the new optimum lies on
// it, where minimising det_i(v) subject to det_j(v) <= det_i(v) (j < i) and
// the disc is a 2D LP with the linear objective n_i . v.  Writes the point.
// Plane offsets are taken relative to s, the agent's own velocity:
// c'_i = det(d_i, P_i - s).  ORCA lines pass near s (through it when
// f = 0), so these offsets are small and exact where they vanish; offsets
// relative to the origin would carry |P| times the FP32 rounding, which the
// bisector of two nearly parallel planes divides by |n_j - n_i| (a vehicle
// at full speed among pedestrians: ten lines through v_A, 5e-3 apart in
// angle, put the vertex 1e-3 m/s off).  Points are in ordinary coordinates.
// In exact arithmetic each sub-problem is non-empty; when rounding makes one
// look empty (a bisector that misses the disc, or a 1D interval emptier than
// the allowance) the step keeps its current point, and *fallback is set: the
// result is then only an upper bound of t*.
__device__ __forceinline__ float lp3_min_penetration(const float4* __restrict__ L, int stride,
                                                     int n, float vmax, float sx, float sy,
                                                     float& vx, float& vy, int& work,
                                                     uint32_t& act, bool* fallback = nullptr) {
    const float tol = lp_tol(vmax);
    // det(d, P - s)
    auto cof = [&](float4 l) { return l.z * (l.y - sy) - l.w * (l.x - sx); };
    float4 l0 = L[0];
    vx = -l0.w * vmax;
    vy = l0.z * vmax;
    act = act_pack(ACT_VERTEX, true, 1, 0, 0, 0);
    float t = penetration(l0, vx, vy);
    for (int i = 1; i < n; ++i) {
        float4 li = L[i * stride];
        if (penetration(li, vx, vy) <= t) continue;
        float nix = -li.w, niy = li.z;   // objective: maximise n_i . v
        float cx = vmax * nix, cy = vmax * niy;
        const float ci = cof(li);
        uint32_t ai = act_pack(ACT_VERTEX, true, 1, i, 0, 0);
        for (int j = 0; j < i; ++j) {
            ++work;
            const float4 lj = L[j * stride];
            // is plane j above plane i at the current point?
            // (n_j - n_i) . (c - s) < c'_j - c'_i, tested before the bisector is built
            const float ax = li.w - lj.w, ay = lj.z - li.z;   // n_j - n_i
            const float beta = cof(lj) - ci;
            if (beta - (ax * (cx - sx) + ay * (cy - sy)) <= 0.0f) continue;
            // bisector {det_j = det_i}: (n_j - n_i) . (v - s) = c'_j - c'_i, as a
            // line through its point closest to s, B' relative to s, with
            // direction e (admissible side det_j <= det_i on its left)
            const float a2 = ax * ax + ay * ay;
            if (a2 <= 1e-12f) continue;   // same direction: one plane dominates
            const float sc = __fdividef(beta, a2);
            const float inv = rsqrtf(a2);
            const float bpx = ax * sc, bpy = ay * sc;
            const float ex = ay * inv, ey = -ax * inv;
            const float bx = bpx + sx, by = bpy + sy;
            float dot = bx * ex + by * ey;
            float disc = dot * dot + vmax * vmax - (bx * bx + by * by);
            if (disc < -tol * (1.0f + vmax)) {
                if (fallback) *fallback = true;
                continue;
            }
            float sq = sqrtf(fmaxf(disc, 0.0f));
            float tl = -dot - sq, tr = -dot + sq;
            int kl = -1, kr = -1;
            bool ok = true;
            for (int jj = 0; jj < j; ++jj) {
                work += 2;   // a bisector and a 1D bound
                // plane jj stays below plane i: (n_jj - n_i) . (v - s) >= c'_jj - c'_i,
                // on the bisector at v = s + B' + t e: t (a . e) >= (c'_jj - c'_i) - a . B'
                const float4 lk = L[jj * stride];
                const float kx = li.w - lk.w, ky = lk.z - li.z;   // n_jj - n_i
                if (kx * kx + ky * ky <= 1e-12f) continue;        // same direction
                const float bk = cof(lk) - ci;
                const float den = kx * ex + ky * ey;
                const float num = bk - (kx * bpx + ky * bpy);
                if (den == 0.0f) {
                    if (num > tol) { ok = false; break; }
                    continue;
                }
                const float tt = __fdividef(num, den);
                if (den < 0.0f) {
                    if (tt < tr) kr = jj;
                    tr = fminf(tr, tt);
                } else {
                    if (tt > tl) kl = jj;
                    tl = fmaxf(tl, tt);
                }
                if (tl > tr + tol) { ok = false; break; }
            }
            if (!ok) {   // empty only through rounding: keep the point
                if (fallback) *fallback = true;
                continue;
            }
            const bool right = nix * ex + niy * ey > 0.0f;
            float tt = right ? tr : tl;
            const int kb = right ? kr : kl;
            cx = bx + tt * ex;
            cy = by + tt * ey;
            ai = kb >= 0 ? act_pack(ACT_VERTEX, false, 3, i, j, kb)
                         : act_pack(ACT_VERTEX, true, 2, i, j, 0);
        }
        vx = cx;
        vy = cy;
        act = ai;
        t = penetration(li, vx, vy);
    }
    float tm = -CUDART_INF_F;
    for (int i = 0; i < n; ++i) tm = fmaxf(tm, penetration(L[i * stride], vx, vy));
    return tm;
}

// The set of least-penetration velocities is one point unless two of the
// half-planes attaining t* are exactly opposite (a valley between two
// neighbours); then it is the part of the valley's mid-line that keeps every
// other half-plane within t* and the disc, and the result is its point
// closest to v_pref.  Returns true and writes that point for a valley.
__device__ __forceinline__ bool valley_tie_break(const float4* __restrict__ L, int stride,
                                                 int n, float t3, float vmax, float vpx,
                                                 float vpy, float v3x, float v3y, float& ox,
                                                 float& oy, int& work, uint32_t& act) {
    const float atol = 1e-5f * (1.0f + fabsf(t3));
    // the lines attaining t* (within atol), then the first exactly opposite
    // pair among them, in the order (i, j) of the line indices
    unsigned long long amask = 0ull;
    for (int i = 0; i < n; ++i)
        if (!(penetration(L[i * stride], v3x, v3y) < t3 - atol)) amask |= 1ull << i;
    int vi = -1, vj = -1;
    for (unsigned long long m = amask; m != 0ull && vi < 0; m &= m - 1ull) {
        const int i = __ffsll((long long)m) - 1;
        const float4 li = L[i * stride];
        for (unsigned long long m2 = m & (m - 1ull); m2 != 0ull; m2 &= m2 - 1ull) {
            const int j = __ffsll((long long)m2) - 1;
            ++work;
            const float4 lj = L[j * stride];
            if (fabsf(li.z * lj.w - li.w * lj.z) > 2e-7f || li.z * lj.z + li.w * lj.w >= 0.0f)
                continue;
            vi = i;
            vj = j;
            break;
        }
    }
    if (vi < 0) return false;
    float4 m;
    if (!bisector(L[vi * stride], L[vj * stride], m)) return false;
    const float tol = lp_tol(vmax);
    const float dot = m.x * m.z + m.y * m.w;
    const float disc = dot * dot + vmax * vmax - (m.x * m.x + m.y * m.y);
    if (disc < -tol * (1.0f + vmax)) return false;
    const float sq = sqrtf(fmaxf(disc, 0.0f));
    float tl = -dot - sq, tr = -dot + sq;
    const float T = t3 + 1e-6f * (1.0f + fabsf(t3));
    int kl = -1, kr = -1;
    for (int k = 0; k < n; ++k) {
        if (k == vi || k == vj) continue;
        ++work;
        const float4 lk = L[k * stride];
        // det(d_k, P_k - (M + s e)) <= T  <=>  s det(e, d_k) <= T - det(d_k, P_k - M)
        const float den = m.z * lk.w - m.w * lk.z;
        const float num = T - (lk.z * (lk.y - m.y) - lk.w * (lk.x - m.x));
        if (den == 0.0f) {
            if (num < -tol) return false;
            continue;
        }
        const float s = __fdividef(num, den);
        if (den > 0.0f) {
            if (s < tr) kr = k;
            tr = fminf(tr, s);
        } else {
            if (s > tl) kl = k;
            tl = fmaxf(tl, s);
        }
    }
    if (tl > tr + tol) return false;
    const float s0 = m.z * (vpx - m.x) + m.w * (vpy - m.y);
    const float s = fminf(fmaxf(s0, tl), tr);
    const int kb = (s0 > tr) ? kr : ((s0 < tl) ? kl : -2);
    act = kb >= 0   ? act_pack(ACT_VERTEX, false, 3, vi, vj, kb)
          : kb == -1 ? act_pack(ACT_VERTEX, true, 2, vi, vj, 0)
                     : act_pack(ACT_VALLEY, false, 2, vi, vj, 0);
    ox = m.x + s * m.z;
    oy = m.y + s * m.w;
    return true;
}

// The velocity of one agent (paper Sec. 3): the admissible velocity closest
// to v_pref, else the velocity of least penetration.  Lines are consumed in
// the order given.  Returns 1 when the half-planes were infeasible.
// The least-penetration LP runs first.  Its t* (offsets relative to the
// agent's velocity) is accurate to well below 0.1 tol, so t* above that,
// with no rounding fallback in any step, means no velocity is admissible
// (the definition, t* > 0) and the 2D LP is skipped.  Otherwise the 2D LP
// decides, its emptiness allowance covering the rounding of exactly
// feasible problems such as f = 0 half-planes all through the agent's own
// velocity on the speed circle.  In dense crowds most agents take the first
// branch, which saves their 2D LP.
__device__ __forceinline__ int solve_velocity(const float4* __restrict__ L, int stride, int n,
                                              float vmax, float vpx, float vpy, float sx,
                                              float sy, float& vx, float& vy, float& tstar,
                                              int& work, uint32_t& act) {
    tstar = 0.0f;
    if (n == 0) return lp2_project(L, stride, n, vmax, vpx, vpy, vx, vy, work, act) == n ? 0 : 1;
    float v3x, v3y;
    uint32_t act3;
    bool fallback = false;
    const float t3 =
        lp3_min_penetration(L, stride, n, vmax, sx, sy, v3x, v3y, work, act3, &fallback);
    if ((t3 <= 0.1f * lp_tol(vmax) || fallback) &&
        lp2_project(L, stride, n, vmax, vpx, vpy, vx, vy, work, act) == n)
        return 0;
    act = act3;
    tstar = t3;
    vx = v3x;
    vy = v3y;
    float ox, oy;
    if (valley_tie_break(L, stride, n, t3, vmax, vpx, vpy, v3x, v3y, ox, oy, work, act)) {
        vx = ox;
        vy = oy;
    }
    return 1;
}

// ---------------------------------------------------------------------------
// The paper's batch-LP load balancing, for comparison (Sec. 3, LP
// paragraphs): each thread owns one agent's LP and scans its constraints
// incrementally; when the current optimum violates constraint i, the re-solve
// on line i is split into work units, one per earlier constraint j, and every
// thread of the block takes its share of all pending units, whether or not its
// own LP needs a re-solve.  The block runs the scan in lockstep over i.  Each
// unit yields one bound of line i's interval, merged with shared-memory
// atomics; min and max are exact, so the interval equals the per-thread
// solver's up to how the compiler contracts the bound's multiply-adds.
// Every agent first runs the per-thread least-penetration LP and makes the
// per-thread scheme's feasibility decision (solve_velocity); agents left
// undecided share the lockstep 2D LP, and those whose 2D LP is empty take
// the least-penetration result.
// ---------------------------------------------------------------------------

// order-preserving map of floats to ints (for atomic min/max)
__device__ __forceinline__ int f2o(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

constexpr int kWorkUnitMaxBlock = 128;

// All threads of the block must call this (inactive ones with n = 0).
// lines_base is the block's line array (agent a, line j at [j * B + a]).
__device__ __forceinline__ int solve_velocity_work_units(const float4* __restrict__ lines_base,
                                                         int n, float vmax, float vpx,
                                                         float vpy, float sx, float sy,
                                                         float& vx, float& vy, float& tstar,
                                                         int& work) {
    __shared__ int s_tl[kWorkUnitMaxBlock], s_tr[kWorkUnitMaxBlock];
    __shared__ int s_empty[kWorkUnitMaxBlock], s_list[kWorkUnitMaxBlock];
    __shared__ float s_tol[kWorkUnitMaxBlock];
    __shared__ int s_n, s_kmax;
    const int tid = threadIdx.x, B = blockDim.x;
    const float4* L = lines_base + tid;
    const float tol = lp_tol(vmax);
    tstar = 0.0f;
    const float vp2 = vpx * vpx + vpy * vpy;
    if (vp2 > vmax * vmax) {
        const float sc = vmax / sqrtf(vp2);
        vx = vpx * sc;
        vy = vpy * sc;
    } else {
        vx = vpx;
        vy = vpy;
    }
    s_tol[tid] = tol;
    if (tid == 0) {
        s_kmax = 0;
        s_n = 0;
    }
    __syncthreads();
    atomicMax(&s_kmax, n);
    __syncthreads();
    const int kmax = s_kmax;
    // the least-penetration LP first, with the per-thread scheme's decision
    // (solve_velocity): a t* above 0.1 tol without rounding fallback is
    // infeasible, and that agent only takes part in the block's lockstep
    float v3x = 0.0f, v3y = 0.0f, t3 = 0.0f;
    uint32_t act = 0u;
    bool live = true;
    if (n > 0) {
        bool fallback = false;
        t3 = lp3_min_penetration(L, B, n, vmax, sx, sy, v3x, v3y, work, act, &fallback);
        live = !(t3 > 0.1f * tol && !fallback);
    }
    for (int i = 0; i < kmax; ++i) {
        bool need = false;
        float4 li = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (live && i < n) {
            li = L[i * B];
            need = penetration(li, vx, vy) > 0.0f;
        }
        if (need) {
            const float dot = li.x * li.z + li.y * li.w;
            const float disc = dot * dot + vmax * vmax - (li.x * li.x + li.y * li.y);
            const float sq = sqrtf(fmaxf(disc, 0.0f));
            s_tl[tid] = f2o(-dot - sq);
            s_tr[tid] = f2o(-dot + sq);
            s_empty[tid] = disc < -tol * (1.0f + vmax) ? 1 : 0;
            s_list[atomicAdd(&s_n, 1)] = tid;
        }
        __syncthreads();
        const int units = s_n * i;   // one unit = (agent needing a re-solve, earlier line)
        for (int w = tid; w < units; w += B) {
            const int q = w / i;
            const int a = s_list[q], j = w - q * i;
            const float4 la = lines_base[i * B + a], lj = lines_base[j * B + a];
            const float den = la.z * lj.w - la.w * lj.z;                     // det(d_i, d_j)
            const float num = lj.z * (la.y - lj.y) - lj.w * (la.x - lj.x);   // det(d_j, P_i - P_j)
            if (den == 0.0f) {
                if (num < -s_tol[a]) atomicOr(&s_empty[a], 1);
            } else {
                const float t = __fdividef(num, den);
                if (den > 0.0f) atomicMin(&s_tr[a], f2o(t));
                else atomicMax(&s_tl[a], f2o(t));
            }
        }
        work += units > 0 ? (units + B - 1) / B : 0;
        __syncthreads();
        if (need) {
            const float tl = o2f(s_tl[tid]), tr = o2f(s_tr[tid]);
            if (s_empty[tid] || tl > tr + tol) {
                live = false;
            } else {
                const float t0 = li.z * (vpx - li.x) + li.w * (vpy - li.y);
                const float t = fminf(fmaxf(t0, tl), tr);
                vx = li.x + t * li.z;
                vy = li.y + t * li.w;
            }
        }
        if (tid == 0) s_n = 0;
        __syncthreads();
    }
    if (live) return 0;
    tstar = t3;
    vx = v3x;
    vy = v3y;
    float ox, oy;
    if (valley_tie_break(L, B, n, t3, vmax, vpx, vpy, v3x, v3y, ox, oy, work, act)) {
        vx = ox;
        vy = oy;
    }
    return 1;
}

// ---------------------------------------------------------------------------
// Active-set enumeration, for comparison: every point where the optimum can
// sit is built and tested against all half-planes and the speed disc, in an
// order that depends only on the number of lines.
//   Admissible velocity: v_pref (its radial projection when faster than
//   vmax); on every line the projection of v_pref clamped to the line's
//   chord of the disc, and both chord ends; the crossing of every pair of
//   lines.  The admissible candidate nearest v_pref is the optimum (Sec. 3,
//   LP paragraphs), since the optimum of the projection onto a convex
//   polygon cut by a disc is one of these points.
//   Least penetration, when no candidate is admissible (Sec. 3,
//   infeasible-set paragraph): t* = min over the disc of max_i det_i(v) is
//   reached where three of {the planes det_i, the disc's rim} are active:
//   the rim point of least penetration of one half-plane, the rim points
//   where two half-planes penetrate equally, and the points where three do.
//   The candidate with the smallest largest penetration wins, then the
//   valley tie-break.
// O(k^3) work per agent, against O(k^2) for the incremental scheme.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float max_penetration(const float4* __restrict__ L, int stride, int n,
                                                 float x, float y) {
    float t = -CUDART_INF_F;
    for (int l = 0; l < n; ++l) t = fmaxf(t, penetration(L[l * stride], x, y));
    return t;
}

__device__ __forceinline__ int solve_velocity_enumeration(const float4* __restrict__ L,
                                                          int stride, int n, float vmax,
                                                          float vpx, float vpy, float& vx,
                                                          float& vy, float& tstar, int& work) {
    const float tol = lp_tol(vmax);
    // the disc, widened by the rounding of points built on its rim
    const float r2 = vmax * vmax + 2.0f * tol * vmax;
    float bd = CUDART_INF_F, bx = 0.0f, by = 0.0f;
    auto offer = [&](float x, float y) {
        if (x * x + y * y > r2) return;
        if (max_penetration(L, stride, n, x, y) > tol) return;
        const float dx = x - vpx, dy = y - vpy;
        const float d = dx * dx + dy * dy;
        if (d < bd) {
            bd = d;
            bx = x;
            by = y;
        }
    };
    {
        const float vp2 = vpx * vpx + vpy * vpy;
        if (vp2 > vmax * vmax) {
            const float sc = vmax / sqrtf(vp2);
            offer(vpx * sc, vpy * sc);
        } else {
            offer(vpx, vpy);
        }
    }
    for (int i = 0; i < n; ++i) {
        const float4 li = L[i * stride];
        const float dot = li.x * li.z + li.y * li.w;
        const float disc = dot * dot + vmax * vmax - (li.x * li.x + li.y * li.y);
        if (disc < -tol * (1.0f + vmax)) continue;   // the line misses the disc
        const float sq = sqrtf(fmaxf(disc, 0.0f));
        const float tl = -dot - sq, tr = -dot + sq;
        const float t0 = li.z * (vpx - li.x) + li.w * (vpy - li.y);
        const float t = fminf(fmaxf(t0, tl), tr);
        offer(li.x + t * li.z, li.y + t * li.w);
        offer(li.x + tl * li.z, li.y + tl * li.w);
        offer(li.x + tr * li.z, li.y + tr * li.w);
        for (int j = 0; j < i; ++j) {
            const float4 lj = L[j * stride];
            const float den = li.z * lj.w - li.w * lj.z;                     // det(d_i, d_j)
            if (den == 0.0f) continue;
            const float num = lj.z * (li.y - lj.y) - lj.w * (li.x - lj.x);   // det(d_j, P_i - P_j)
            const float tt = __fdividef(num, den);
            offer(li.x + tt * li.z, li.y + tt * li.w);
        }
    }
    work += n * (n + 1) / 2;
    tstar = 0.0f;
    if (bd < CUDART_INF_F) {
        vx = bx;
        vy = by;
        return 0;
    }
    float bt = CUDART_INF_F;
    auto offer3 = [&](float x, float y) {
        if (x * x + y * y > r2) return;
        const float t = max_penetration(L, stride, n, x, y);
        if (t < bt) {
            bt = t;
            bx = x;
            by = y;
        }
    };
    for (int i = 0; i < n; ++i) {
        const float4 li = L[i * stride];
        const float ci = li.z * li.y - li.w * li.x;   // c = det(d, P), pen(v) = c - n . v
        offer3(-li.w * vmax, li.z * vmax);            // vmax n_i, n = (-d_y, d_x)
        for (int j = 0; j < i; ++j) {
            const float4 lj = L[j * stride];
            float4 bij;
            if (!bisector(li, lj, bij)) continue;
            const float dot = bij.x * bij.z + bij.y * bij.w;
            const float disc = dot * dot + vmax * vmax - (bij.x * bij.x + bij.y * bij.y);
            if (disc >= 0.0f) {
                const float sq = sqrtf(disc);
                offer3(bij.x + (-dot - sq) * bij.z, bij.y + (-dot - sq) * bij.w);
                offer3(bij.x + (-dot + sq) * bij.z, bij.y + (-dot + sq) * bij.w);
            }
            // pen_i = pen_j = pen_m: (n_j - n_i) . v = c_j - c_i and
            // (n_m - n_i) . v = c_m - c_i, by Cramer's rule
            const float a1x = li.w - lj.w, a1y = lj.z - li.z;
            const float b1 = (lj.z * lj.y - lj.w * lj.x) - ci;
            const float n1 = sqrtf(a1x * a1x + a1y * a1y);
            for (int m = 0; m < j; ++m) {
                const float4 lm = L[m * stride];
                const float a2x = li.w - lm.w, a2y = lm.z - li.z;
                const float b2 = (lm.z * lm.y - lm.w * lm.x) - ci;
                const float det = a1x * a2y - a1y * a2x;
                // sine between the two normals: skip (near-)parallel pairs
                if (fabsf(det) < 1e-6f * n1 * sqrtf(a2x * a2x + a2y * a2y)) continue;
                offer3((b1 * a2y - b2 * a1y) / det, (a1x * b2 - a2x * b1) / det);
            }
        }
    }
    work += n * (n - 1) * (n + 1) / 6;
    tstar = bt;
    vx = bx;
    vy = by;
    float ox, oy;
    uint32_t act = 0u;
    if (valley_tie_break(L, stride, n, bt, vmax, vpx, vpy, bx, by, ox, oy, work, act)) {
        vx = ox;
        vy = oy;
    }
    return 1;
}

// ---------------------------------------------------------------------------
// Warp-cooperative LP, for comparison: a warp solves the LPs of its 32
// agents one after another, and within each 1D sub-problem (a line against
// the earlier lines, or a bisector against the earlier planes) lane j takes
// constraint j.  The interval ends are merged by warp reductions on
// order-preserving integer images of the bounds (exact min and max), so the
// result equals the per-thread LP's up to how the compiler contracts the
// bounds' multiply-adds.  Every lane of the warp must call it (lanes without
// an agent with n = 0).  lines_base is the block's line array (agent a,
// line j at [j * B + a]); warp0 is the block index of the warp's lane 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_fmax(float x) {
    return o2f(__reduce_max_sync(0xffffffffu, f2o(x)));
}
__device__ __forceinline__ float warp_fmin(float x) {
    return o2f(__reduce_min_sync(0xffffffffu, f2o(x)));
}

// 1D problem on line li against lines 0..i-1 of La: the interval [tl, tr]
// of li inside the disc and the earlier half-planes; false when empty.
__device__ __forceinline__ bool warp_lp1_interval(const float4* __restrict__ La, int B, int i,
                                                  float4 li, float vmax, float tol, float& tl,
                                                  float& tr) {
    const float dot = li.x * li.z + li.y * li.w;
    const float disc = dot * dot + vmax * vmax - (li.x * li.x + li.y * li.y);
    if (disc < -tol * (1.0f + vmax)) return false;
    const float sq = sqrtf(fmaxf(disc, 0.0f));
    float lo = -dot - sq, hi = -dot + sq;
    bool empty = false;
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < i; j0 += 32) {
        const int j = j0 + lane;
        float blo = -CUDART_INF_F, bhi = CUDART_INF_F;
        if (j < i) {
            const float4 lj = La[j * B];
            const float den = li.z * lj.w - li.w * lj.z;                     // det(d_i, d_j)
            const float num = lj.z * (li.y - lj.y) - lj.w * (li.x - lj.x);   // det(d_j, P_i - P_j)
            if (den == 0.0f) {
                empty |= num < -tol;
            } else {
                const float t = __fdividef(num, den);
                if (den > 0.0f) bhi = t;
                else blo = t;
            }
        }
        lo = fmaxf(lo, warp_fmax(blo));
        hi = fminf(hi, warp_fmin(bhi));
    }
    if (__any_sync(0xffffffffu, empty)) return false;
    tl = lo;
    tr = hi;
    return !(lo > hi + tol);
}

__device__ __forceinline__ int solve_velocity_warp(const float4* __restrict__ lines_base,
                                                   int warp0, int n_own, float vmax_own,
                                                   float vpx_own, float vpy_own, float& vx,
                                                   float& vy, float& tstar, int& work) {
    const int lane = threadIdx.x & 31, B = blockDim.x;
    int infeasible = 0;
    vx = vy = tstar = 0.0f;
    for (int a = 0; a < 32; ++a) {
        const int n = __shfl_sync(0xffffffffu, n_own, a);
        const float vmax = __shfl_sync(0xffffffffu, vmax_own, a);
        const float vpx = __shfl_sync(0xffffffffu, vpx_own, a);
        const float vpy = __shfl_sync(0xffffffffu, vpy_own, a);
        const float4* La = lines_base + warp0 + a;
        const float tol = lp_tol(vmax);
        // ---- projection of v_pref (incremental over the lines) ----
        float ox, oy;
        const float vp2 = vpx * vpx + vpy * vpy;
        if (vp2 > vmax * vmax) {
            const float sc = vmax / sqrtf(vp2);
            ox = vpx * sc;
            oy = vpy * sc;
        } else {
            ox = vpx;
            oy = vpy;
        }
        bool feasible = true;
        for (int i = 0; i < n && feasible; ++i) {
            const float4 li = La[i * B];
            if (penetration(li, ox, oy) <= 0.0f) continue;
            float tl, tr;
            work += (i + 31) / 32;
            if (!warp_lp1_interval(La, B, i, li, vmax, tol, tl, tr)) {
                feasible = false;
                break;
            }
            const float t0 = li.z * (vpx - li.x) + li.w * (vpy - li.y);
            const float t = fminf(fmaxf(t0, tl), tr);
            ox = li.x + t * li.z;
            oy = li.y + t * li.w;
        }
        float ts = 0.0f;
        if (!feasible) {
            // ---- least penetration (incremental LP in (v, t)) ----
            const float4 l0 = La[0];
            float cx0 = -l0.w * vmax, cy0 = l0.z * vmax;
            float t = penetration(l0, cx0, cy0);
            for (int i = 1; i < n; ++i) {
                const float4 li = La[i * B];
                if (penetration(li, cx0, cy0) <= t) continue;
                const float nix = -li.w, niy = li.z;
                float cx = vmax * nix, cy = vmax * niy;
                const float ci = li.z * li.y - li.w * li.x;
                for (int j = 0; j < i; ++j) {
                    const float4 lj = La[j * B];
                    {
                        const float ax = li.w - lj.w, ay = lj.z - li.z;
                        const float beta = (lj.z * lj.y - lj.w * lj.x) - ci;
                        if (beta - (ax * cx + ay * cy) <= 0.0f) continue;
                    }
                    float4 bj;
                    if (!bisector(li, lj, bj)) continue;
                    const float dot = bj.x * bj.z + bj.y * bj.w;
                    const float disc = dot * dot + vmax * vmax - (bj.x * bj.x + bj.y * bj.y);
                    if (disc < -tol * (1.0f + vmax)) continue;
                    const float sq = sqrtf(fmaxf(disc, 0.0f));
                    float lo = -dot - sq, hi = -dot + sq;
                    bool bad = false;
                    work += (j + 31) / 32;
                    for (int k0 = 0; k0 < j; k0 += 32) {
                        const int jj = k0 + lane;
                        float blo = -CUDART_INF_F, bhi = CUDART_INF_F;
                        if (jj < j) {
                            const float4 lk = La[jj * B];
                            const float ax = li.w - lk.w, ay = lk.z - li.z;   // n_jj - n_i
                            if (ax * ax + ay * ay > 1e-12f) {
                                const float beta = (lk.z * lk.y - lk.w * lk.x) - ci;
                                const float den = ax * bj.z + ay * bj.w;
                                const float num = beta - (ax * bj.x + ay * bj.y);
                                if (den == 0.0f) {
                                    bad |= num > tol;
                                } else {
                                    const float tt = __fdividef(num, den);
                                    if (den < 0.0f) bhi = tt;
                                    else blo = tt;
                                }
                            }
                        }
                        lo = fmaxf(lo, warp_fmax(blo));
                        hi = fminf(hi, warp_fmin(bhi));
                    }
                    if (__any_sync(0xffffffffu, bad) || lo > hi + tol) continue;
                    const bool right = nix * bj.z + niy * bj.w > 0.0f;
                    const float tt = right ? hi : lo;
                    cx = bj.x + tt * bj.z;
                    cy = bj.y + tt * bj.w;
                }
                cx0 = cx;
                cy0 = cy;
                t = penetration(li, cx0, cy0);
            }
            float tm = -CUDART_INF_F;
            for (int i = 0; i < n; ++i) tm = fmaxf(tm, penetration(La[i * B], cx0, cy0));
            ts = tm;
            ox = cx0;
            oy = cy0;
            float vx2, vy2;
            uint32_t act = 0u;
            int w2 = 0;
            if (valley_tie_break(La, B, n, tm, vmax, vpx, vpy, cx0, cy0, vx2, vy2, w2, act)) {
                ox = vx2;
                oy = vy2;
            }
        }
        if (lane == a) {
            vx = ox;
            vy = oy;
            tstar = ts;
            infeasible = feasible ? 0 : 1;
        }
    }
    return infeasible;
}

}  // namespace orca
