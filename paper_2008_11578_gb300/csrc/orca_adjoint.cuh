// orca_adjoint.cuh -- reverse-mode derivative of one ORCA step (FP32).
//
// One step maps the state (p_t, v_t) and the preferred-velocity offset
// delta_t to v_{t+1} = LP(lines(p_t, v_t), v_pref(p_t, goal) + delta_t) and
// p_{t+1} = p_t + dt v_{t+1}.  Its adjoint, per agent A:
//   vbar*  = vbar_{t+1}[A] + dL/dv_{t+1}[A] + dt pbar_{t+1}[A]
//   pbar_t[A] += pbar_{t+1}[A]
//   LP: vbar* -> (v_pref, active lines) by the implicit function on the
//       recorded active set; discrete choices (neighbours, active set, leg,
//       cut-off or overlap construction, waypoint) carry no gradient
//   lines: (Pbar, dbar) -> own p, v and the neighbour's p, v (atomics)
//   v_pref: -> own p, delta_t, and the current waypoint of a routed agent.
// Only the 1-3 active lines have non-zero cotangents, so the kernel rebuilds
// just those from the recorded state.
#pragma once

#include "orca_kernels.cuh"

namespace orca {

// Backward of orca_line: (Pbar, dbar) of the line of A against B, given the
// construction the forward took, into the cotangents of p_A, v_A, p_B, v_B.
__device__ __forceinline__ void orca_line_backward(
    float pax, float pay, float vax, float vay, float ra, float pbx, float pby, float vbx,
    float vby, float rb, float f, float inv_tau, float inv_dt, bool overlap, bool cap,
    float4 bar, float& gpax, float& gpay, float& gvax, float& gvay, float& gpbx, float& gpby,
    float& gvbx, float& gvby) {
    const float qx = pbx - pax, qy = pby - pay;
    const float wrx = vax - vbx, wry = vay - vby;
    const float rho = ra + rb;
    float gqx = 0.0f, gqy = 0.0f, gwx = 0.0f, gwy = 0.0f;
    // P = v_A + f u
    gvax += bar.x;
    gvay += bar.y;
    const float ubx = f * bar.x, uby = f * bar.y;
    if (overlap || cap) {
        // u = s h, d = (h_y, -h_x), s = rho T - |w|, h = w / |w|, w = w_rel - q T
        const float T = overlap ? inv_dt : inv_tau;
        const float wx = wrx - qx * T, wy = wry - qy * T;
        const float wl = sqrtf(wx * wx + wy * wy);
        if (wl > 0.0f) {
            const float hx = wx / wl, hy = wy / wl;
            const float s = rho * T - wl;
            const float sbar = ubx * hx + uby * hy;
            const float hbx = s * ubx - bar.w;
            const float hby = s * uby + bar.z;
            const float wlbar = -sbar;
            const float hd = hx * hbx + hy * hby;
            const float wbx = (hbx - hx * hd) / wl + hx * wlbar;
            const float wby = (hby - hy * hd) / wl + hy * wlbar;
            gwx += wbx;
            gwy += wby;
            gqx -= T * wbx;
            gqy -= T * wby;
        }
    } else {
        // legs: d = sg (a, b) / |q|^2 with l = sqrt(|q|^2 - rho^2);
        // u = (w_rel . d) d - w_rel
        const float qq = qx * qx + qy * qy;
        const float l = sqrtf(fmaxf(leg_l2(qx, qy, ra, rb, qq, rho * rho), 0.0f));
        const float iq = 1.0f / qq;
        const bool left = leg_left(pax, pay, pbx, pby, vax, vay, vbx, vby);
        const float sg = left ? 1.0f : -1.0f;
        const float a = left ? qx * l - qy * rho : qx * l + qy * rho;
        const float b = left ? qx * rho + qy * l : qy * l - qx * rho;
        const float dx = sg * a * iq, dy = sg * b * iq;
        const float pr = wrx * dx + wry * dy;
        const float prbar = ubx * dx + uby * dy;
        const float ddx = bar.z + pr * ubx + prbar * wrx;
        const float ddy = bar.w + pr * uby + prbar * wry;
        gwx += prbar * dx - ubx;
        gwy += prbar * dy - uby;
        const float abar = sg * ddx * iq, bbar = sg * ddy * iq;
        float qqbar = -(ddx * dx + ddy * dy) * iq;
        const float lbar = abar * qx + bbar * qy;
        if (left) {
            gqx += abar * l + bbar * rho;
            gqy += -abar * rho + bbar * l;
        } else {
            gqx += abar * l - bbar * rho;
            gqy += abar * rho + bbar * l;
        }
        if (l > 0.0f) qqbar += 0.5f * lbar / l;
        gqx += 2.0f * qqbar * qx;
        gqy += 2.0f * qqbar * qy;
    }
    // q = p_B - p_A, w_rel = v_A - v_B
    gpax -= gqx;
    gpay -= gqy;
    gpbx += gqx;
    gpby += gqy;
    gvax += gwx;
    gvay += gwy;
    gvbx -= gwx;
    gvby -= gwy;
}

// Backward of v_pref = (g - p) min(vmax / |g - p|, 1/dt): the cotangent of
// e = g - p (the caller adds it to g and subtracts it from p).
__device__ __forceinline__ float2 vpref_backward(float px, float py, float gx, float gy,
                                                 float vmax, float inv_dt, float vpbx,
                                                 float vpby) {
    const float ex = gx - px, ey = gy - py;
    const float gl = sqrtf(ex * ex + ey * ey);
    if (!(gl > 0.0f)) return make_float2(0.0f, 0.0f);
    const float sc = vmax / gl;
    if (sc < inv_dt) {
        const float hx = ex / gl, hy = ey / gl;
        const float dot = hx * vpbx + hy * vpby;
        return make_float2(sc * (vpbx - hx * dot), sc * (vpby - hy * dot));
    }
    return make_float2(inv_dt * vpbx, inv_dt * vpby);
}

__device__ __forceinline__ float det3(float a00, float a01, float a02, float a10, float a11,
                                      float a12, float a20, float a21, float a22) {
    return a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
           a02 * (a10 * a21 - a11 * a20);
}

// Cotangents of the LP result v* = (vx, vy) with respect to v_pref and the
// active lines la[m] = (P, d) of the recorded active set `act`:
//   projection with no line:   v = v_pref, or vmax v_pref / |v_pref|
//   projection onto one line:  v = P + (d . (v_pref - P)) d
//   valley:                    projection onto {(n_b - n_a) . v = c_b - c_a}
//   one plane on the circle:   v = vmax n_a
//   vertices (two boundaries in 2D, three in (v, t)): implicit function of
//     F_line = det(d, P - v) [- t] = 0 and F_circle = (|v|^2 - vmax^2) / 2 = 0,
//     y = J^-T (vbar [, 0]), Pbar = y (d_y, -d_x), dbar = -y (P_y - v_y, v_x - P_x)
// with n = (-d_y, d_x) and c = det(d, P).  Degenerate systems give zero.
__device__ __forceinline__ void lp_backward(uint32_t act, const float4* la, float vmax,
                                            float vpx, float vpy, float vx, float vy,
                                            float vbx, float vby, float& vpbx, float& vpby,
                                            float4* lbar) {
    vpbx = vpby = 0.0f;
#pragma unroll
    for (int m = 0; m < 3; ++m) lbar[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const uint32_t kind = act_kind(act);
    const bool circ = act_circle(act);
    const int nl = act_nlines(act);
    if (kind == ACT_PROJ && nl == 0) {
        if (!circ) {
            vpbx = vbx;
            vpby = vby;
        } else {
            const float ul = sqrtf(vpx * vpx + vpy * vpy);
            if (ul > 0.0f) {
                const float hx = vpx / ul, hy = vpy / ul;
                const float dot = hx * vbx + hy * vby;
                vpbx = vmax / ul * (vbx - hx * dot);
                vpby = vmax / ul * (vby - hy * dot);
            }
        }
        return;
    }
    if (kind == ACT_PROJ && nl == 1 && !circ) {
        const float4 L = la[0];
        const float ex = vpx - L.x, ey = vpy - L.y;
        const float tau = L.z * ex + L.w * ey;
        const float taub = L.z * vbx + L.w * vby;
        lbar[0] = make_float4(vbx - taub * L.z, vby - taub * L.w, tau * vbx + taub * ex,
                              tau * vby + taub * ey);
        vpbx = taub * L.z;
        vpby = taub * L.w;
        return;
    }
    if (kind == ACT_VALLEY) {
        if (nl != 2) return;
        const float4 A = la[0], B = la[1];
        const float ax = A.w - B.w, ay = B.z - A.z;   // n_b - n_a
        const float beta = (B.z * B.y - B.w * B.x) - (A.z * A.y - A.w * A.x);
        const float a2 = ax * ax + ay * ay;
        if (!(a2 > 1e-12f)) return;
        const float s = (beta - (ax * vpx + ay * vpy)) / a2;
        const float adot = (ax * vbx + ay * vby) / a2;
        vpbx = vbx - ax * adot;
        vpby = vby - ay * adot;
        const float abx = s * vbx - adot * (vpx + 2.0f * s * ax);
        const float aby = s * vby - adot * (vpy + 2.0f * s * ay);
        // n_b += abar, n_a -= abar; c_b += adot, c_a -= adot
        // nbar -> dbar: (dbar_x, dbar_y) += (nbar_y, -nbar_x)
        // cbar -> Pbar: (-cbar d_y, cbar d_x), dbar: (cbar P_y, -cbar P_x)
        lbar[1] = make_float4(-adot * B.w, adot * B.z, aby + adot * B.y, -abx - adot * B.x);
        lbar[0] = make_float4(adot * A.w, -adot * A.z, -aby - adot * A.y, abx + adot * A.x);
        return;
    }
    if (kind == ACT_VERTEX && nl == 1 && circ) {
        const float4 A = la[0];
        (void)A;
        lbar[0] = make_float4(0.0f, 0.0f, vmax * vby, -vmax * vbx);
        return;
    }
    // vertex systems
    float y[3] = {0.0f, 0.0f, 0.0f};
    if (kind == ACT_PROJ) {
        if (nl + (circ ? 1 : 0) != 2) return;
        float J[2][2];
        for (int m = 0; m < nl; ++m) {
            J[m][0] = la[m].w;
            J[m][1] = -la[m].z;
        }
        if (circ) {
            J[1][0] = vx;
            J[1][1] = vy;
        }
        const float det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const float scale = (fabsf(J[0][0]) + fabsf(J[0][1])) * (fabsf(J[1][0]) + fabsf(J[1][1]));
        if (!(fabsf(det) > 1e-7f * scale)) return;
        y[0] = (vbx * J[1][1] - J[1][0] * vby) / det;
        y[1] = (J[0][0] * vby - vbx * J[0][1]) / det;
    } else {
        if (nl + (circ ? 1 : 0) != 3) return;
        float J[3][3];
        for (int m = 0; m < nl; ++m) {
            J[m][0] = la[m].w;
            J[m][1] = -la[m].z;
            J[m][2] = -1.0f;
        }
        if (circ) {
            J[2][0] = vx;
            J[2][1] = vy;
            J[2][2] = 0.0f;
        }
        // J^T y = (vbx, vby, 0) by Cramer's rule on A = J^T
        const float det = det3(J[0][0], J[1][0], J[2][0], J[0][1], J[1][1], J[2][1], J[0][2],
                               J[1][2], J[2][2]);
        float scale = 1.0f;
        for (int r = 0; r < 3; ++r)
            scale *= fabsf(J[r][0]) + fabsf(J[r][1]) + fabsf(J[r][2]);
        if (!(fabsf(det) > 1e-7f * scale)) return;
        const float z0 = vbx, z1 = vby, z2 = 0.0f;
        y[0] = det3(z0, J[1][0], J[2][0], z1, J[1][1], J[2][1], z2, J[1][2], J[2][2]) / det;
        y[1] = det3(J[0][0], z0, J[2][0], J[0][1], z1, J[2][1], J[0][2], z2, J[2][2]) / det;
        y[2] = det3(J[0][0], J[1][0], z0, J[0][1], J[1][1], z1, J[0][2], J[1][2], z2) / det;
    }
    for (int m = 0; m < nl; ++m) {
        const float4 L = la[m];
        lbar[m] = make_float4(y[m] * L.w, -y[m] * L.z, -y[m] * (L.y - vy), -y[m] * (vx - L.x));
    }
}

__device__ __forceinline__ void atomic_add2(float2* p, float x, float y) {
    atomicAdd(&p->x, x);
    atomicAdd(&p->y, y);
}

// Reverse of step t for every agent (caller order), one thread per agent.
// pos/vel: state at the start of step t; nbr/act/wp_used/vnew: recorded by
// the forward recompute of the step.  pbar_next/vbar_next hold the
// cotangents of the state after the step; this step's cotangents accumulate
// (atomically) into pbar_cur/vbar_cur, which start at zero.  The kernel also
// zeroes pbar_spare/vbar_spare, the accumulators of the step before (three
// buffers rotate, so no buffer is cleared while another thread adds to it).
__global__ void __launch_bounds__(128)
adjoint_kernel(int n, SceneDev sc, const float2* __restrict__ pos, const float2* __restrict__ vel,
               const float* __restrict__ rad, const uint8_t* __restrict__ typ,
               const int32_t* __restrict__ nbr, int k_stride, const uint32_t* __restrict__ act,
               const uint8_t* __restrict__ wp_used, const float2* __restrict__ vnew, AgentIn ain,
               const float2* __restrict__ vpd, const float2* __restrict__ pbar_next,
               const float2* __restrict__ vbar_next, const float2* __restrict__ dl_dv,
               float2* __restrict__ pbar_cur, float2* __restrict__ vbar_cur,
               float2* __restrict__ pbar_spare, float2* __restrict__ vbar_spare,
               float2* __restrict__ dvpd, float2* __restrict__ dwp, const int* __restrict__ err) {
    // the replayed records are not valid after a binning error (see solve_kernel)
    if (__ldcg(err) & (ERR_BIT_TIMEOUT | ERR_BIT_STATE)) return;
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= n) return;
    pbar_spare[A] = make_float2(0.0f, 0.0f);
    vbar_spare[A] = make_float2(0.0f, 0.0f);
    const float2 p = pos[A], v = vel[A];
    const float r = rad[A];
    const int ta = typ[A];
    const float vmax = ain.max_speed[A];
    const float2 pn = pbar_next[A];
    float2 vn = vbar_next[A];
    if (dl_dv != nullptr) {
        const float2 e = dl_dv[A];
        vn.x += e.x;
        vn.y += e.y;
    }
    const float vsbx = vn.x + sc.dt * pn.x, vsby = vn.y + sc.dt * pn.y;
    float gpx = pn.x, gpy = pn.y, gvx = 0.0f, gvy = 0.0f;

    // preferred velocity (the forward's formula)
    float2 g = ain.goal[A];
    int rt = -1, wi = 0;
    if (ain.route != nullptr) {
        rt = ain.route[A];
        if (rt >= 0) {
            wi = wp_used[A];
            g = ain.waypoints[(size_t)rt * ain.n_waypoints + wi];
        }
    }
    float vpx = 0.0f, vpy = 0.0f;
    {
        const float gx = g.x - p.x, gy = g.y - p.y;
        const float gl = sqrtf(gx * gx + gy * gy);
        if (gl > 0.0f) {
            const float f = fminf(vmax / gl, sc.inv_dt);
            vpx = gx * f;
            vpy = gy * f;
        }
        if (vpd != nullptr) {
            const float2 dl = vpd[A];
            vpx += dl.x;
            vpy += dl.y;
        }
    }

    // the active lines, rebuilt from the recorded state
    const uint32_t ac = act[A];
    const int nl = act_nlines(ac);
    float4 la[3];
    int lj[3];
    float lf[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        lj[m] = -1;
        lf[m] = 0.0f;
        la[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (m < nl) {
            const int j = nbr[(size_t)A * k_stride + act_line(ac, m)];
            lj[m] = j;
            const float2 pj = pos[j], vj = vel[j];
            const int tb = typ[j];
            lf[m] = tb ? (ta ? sc.f11 : sc.f01) : (ta ? sc.f10 : sc.f00);
            bool cap;
            la[m] = orca_line(p.x, p.y, v.x, v.y, r, pj.x, pj.y, vj.x, vj.y, rad[j], lf[m],
                              sc.inv_tau, sc.inv_dt, act_overlap(ac, m), cap);
        }
    }
    const float2 vs = vnew[A];
    float vpbx, vpby;
    float4 lbar[3];
    lp_backward(ac, la, vmax, vpx, vpy, vs.x, vs.y, vsbx, vsby, vpbx, vpby, lbar);
    if (dvpd != nullptr) dvpd[A] = make_float2(vpbx, vpby);

    const float2 ge = vpref_backward(p.x, p.y, g.x, g.y, vmax, sc.inv_dt, vpbx, vpby);
    gpx -= ge.x;
    gpy -= ge.y;
    if (rt >= 0 && dwp != nullptr)
        atomic_add2(dwp + (size_t)rt * ain.n_waypoints + wi, ge.x, ge.y);

#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (m < nl) {
            const int j = lj[m];
            const float2 pj = pos[j], vj = vel[j];
            float gpbx = 0.0f, gpby = 0.0f, gvbx = 0.0f, gvby = 0.0f;
            orca_line_backward(p.x, p.y, v.x, v.y, r, pj.x, pj.y, vj.x, vj.y, rad[j], lf[m],
                               sc.inv_tau, sc.inv_dt, act_overlap(ac, m), act_cap(ac, m),
                               lbar[m], gpx, gpy, gvx, gvy, gpbx, gpby, gvbx, gvby);
            atomic_add2(pbar_cur + j, gpbx, gpby);
            atomic_add2(vbar_cur + j, gvbx, gvby);
        }
    }
    atomic_add2(pbar_cur + A, gpx, gpy);
    atomic_add2(vbar_cur + A, gvx, gvy);
}

}  // namespace orca
