// Device-side vehicle models: Euler dynamics of Sec. IV-A (eqn:system_eqn,
// s_{t+1} = s_t + dt f_c(s_t, u_t)), their Jacobians for the step-2
// linearisation, and the pose (rho(s), R(s)) of each robot part with its
// state derivatives (y = R(s) x + rho(s), Sec. IV-A).
#pragma once

#include "oca_common.cuh"

namespace oca {

// 2x2 rotation by angle a and its derivative.
template <typename T>
__device__ __forceinline__ void rot2(T a, T R[4], T dR[4]) {
    T c = m_cos(a), s = m_sin(a);
    R[0] = c; R[1] = -s; R[2] = s; R[3] = c;
    dR[0] = -s; dR[1] = -c; dR[2] = c; dR[3] = -s;
}

// ZYX Euler rotation R = Rz(yaw) Ry(pitch) Rx(roll) and dR/d(roll,pitch,yaw).
template <typename T>
__device__ __forceinline__ void rot3(T ph, T th, T ps, T R[9], T dR[3][9]) {
    T cf = m_cos(ph), sf = m_sin(ph), ct = m_cos(th), st = m_sin(th), cp = m_cos(ps), sp = m_sin(ps);
    // closed forms of the product and its three partial derivatives
    R[0] = cp * ct; R[1] = cp * st * sf - sp * cf; R[2] = cp * st * cf + sp * sf;
    R[3] = sp * ct; R[4] = sp * st * sf + cp * cf; R[5] = sp * st * cf - cp * sf;
    R[6] = -st;     R[7] = ct * sf;                R[8] = ct * cf;
    if (dR) {
        // d/droll
        dR[0][0] = 0; dR[0][1] = cp * st * cf + sp * sf; dR[0][2] = -cp * st * sf + sp * cf;
        dR[0][3] = 0; dR[0][4] = sp * st * cf - cp * sf; dR[0][5] = -sp * st * sf - cp * cf;
        dR[0][6] = 0; dR[0][7] = ct * cf;                dR[0][8] = -ct * sf;
        // d/dpitch
        dR[1][0] = -cp * st; dR[1][1] = cp * ct * sf; dR[1][2] = cp * ct * cf;
        dR[1][3] = -sp * st; dR[1][4] = sp * ct * sf; dR[1][5] = sp * ct * cf;
        dR[1][6] = -ct;      dR[1][7] = -st * sf;     dR[1][8] = -st * cf;
        // d/dyaw
        dR[2][0] = -sp * ct; dR[2][1] = -sp * st * sf - cp * cf; dR[2][2] = -sp * st * cf + cp * sf;
        dR[2][3] = cp * ct;  dR[2][4] = cp * st * sf - sp * cf;  dR[2][5] = cp * st * cf + sp * sf;
        dR[2][6] = 0;        dR[2][7] = 0;                       dR[2][8] = 0;
    }
}

// Pose of a part.  Outputs rho[D], R[D*D]; when drho != nullptr also
// drho[D][NS] (row-major) and, for the NROT rotation coordinates, the state
// index ridx[r] and dR/ds_ridx[r] in dR[r][D*D].
template <typename T, int KIND>
__device__ void part_pose(const DevModel<T> &m, int link, const T *off, const T *s, T *rho, T *R,
                          T *drho, T (*dR)[MDims<KIND>::D * MDims<KIND>::D], int *ridx) {
    constexpr int NS = MDims<KIND>::NS;
    if constexpr (MDims<KIND>::D == 2) {
        const int ai = (KIND == 1 && link == 1) ? 4 : 2;
        T Rp[4];
        rot2<T>(s[ai], R, Rp);
        rho[0] = s[0] + R[0] * off[0] + R[1] * off[1];
        rho[1] = s[1] + R[2] * off[0] + R[3] * off[1];
        T hx = 0, hy = 0;
        if (KIND == 1 && link == 1) {
            // trailer frame origin at the hitch, M behind the rear axle
            T ct = m_cos(s[2]), st = m_sin(s[2]);
            rho[0] -= m.p[1] * ct;
            rho[1] -= m.p[1] * st;
            hx = m.p[1] * st;
            hy = -m.p[1] * ct;
        }
        if (drho) {
#pragma unroll
            for (int k = 0; k < 2 * NS; ++k) drho[k] = T(0);
            drho[0 * NS + 0] = T(1);
            drho[1 * NS + 1] = T(1);
            drho[0 * NS + ai] += Rp[0] * off[0] + Rp[1] * off[1];
            drho[1 * NS + ai] += Rp[2] * off[0] + Rp[3] * off[1];
            if (KIND == 1 && link == 1) {
                drho[0 * NS + 2] += hx;
                drho[1 * NS + 2] += hy;
            }
            ridx[0] = ai;
#pragma unroll
            for (int k = 0; k < 4; ++k) dR[0][k] = Rp[k];
        }
    } else {
        T dR3[3][9];
        rot3<T>(s[6], s[7], s[8], R, drho ? dR3 : nullptr);
#pragma unroll
        for (int i = 0; i < 3; ++i) rho[i] = s[i] + R[i * 3 + 0] * off[0] + R[i * 3 + 1] * off[1] + R[i * 3 + 2] * off[2];
        if (drho) {
#pragma unroll
            for (int k = 0; k < 3 * NS; ++k) drho[k] = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                drho[i * NS + i] = T(1);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    drho[i * NS + 6 + a] = dR3[a][i * 3 + 0] * off[0] + dR3[a][i * 3 + 1] * off[1] + dR3[a][i * 3 + 2] * off[2];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ridx[a] = 6 + a;
#pragma unroll
                for (int k = 0; k < 9; ++k) dR[a][k] = dR3[a][k];
            }
        }
    }
}

// Continuous-time dynamics f_c(s, u) and its Jacobians (row-major
// fs[NS][NS], fu[NS][NU]); fs/fu may be null.
template <typename T, int KIND>
__device__ void dynamics(const DevModel<T> &m, const T *s, const T *u, T *f, T *fs, T *fu) {
    constexpr int NS = MDims<KIND>::NS, NU = MDims<KIND>::NU;
    if (fs) for (int k = 0; k < NS * NS; ++k) fs[k] = T(0);
    if (fu) for (int k = 0; k < NS * NU; ++k) fu[k] = T(0);
    if constexpr (KIND == 0 || KIND == 1) {
        // kinematic bicycle, steering entered as path curvature kappa = tan(steer)/L
        const T th = s[2], v = s[3], kap = u[1];
        const T c = m_cos(th), sn = m_sin(th);
        f[0] = v * c;
        f[1] = v * sn;
        f[2] = v * kap;
        f[3] = u[0];
        if (fs) {
            fs[0 * NS + 2] = -v * sn; fs[0 * NS + 3] = c;
            fs[1 * NS + 2] = v * c;   fs[1 * NS + 3] = sn;
            fs[2 * NS + 3] = kap;
        }
        if (fu) {
            fu[2 * NU + 1] = v;
            fu[3 * NU + 0] = T(1);
        }
        if constexpr (KIND == 1) {
            // trailer heading: hitch M behind the rear axle, trailer axle L2 behind it
            const T Mh = m.p[1], L2 = m.p[2];
            const T dpsi = th - s[4];
            const T cd = m_cos(dpsi), sd = m_sin(dpsi);
            f[4] = (v * sd - v * Mh * kap * cd) / L2;
            if (fs) {
                const T dth = (v * cd + v * Mh * kap * sd) / L2;
                fs[4 * NS + 2] = dth;
                fs[4 * NS + 4] = -dth;
                fs[4 * NS + 3] = (sd - Mh * kap * cd) / L2;
            }
            if (fu) fu[4 * NU + 1] = -v * Mh * cd / L2;
        }
    } else {
        const T mass = m.p[0], g = m.p[1], Jx = m.p[2], Jy = m.p[3], Jz = m.p[4];
        const T arm = m.p[5], km = m.p[6];
        T R[9], dR[3][9];
        rot3<T>(s[6], s[7], s[8], R, fs ? dR : nullptr);
        const T thrust = mass * g + u[0] + u[1] + u[2] + u[3];
        const T p = s[9], q = s[10], r = s[11];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            f[i] = s[3 + i];
            f[3 + i] = R[i * 3 + 2] * thrust / mass;
        }
        f[5] -= g;
        const T cf = m_cos(s[6]), sf = m_sin(s[6]), ct = m_cos(s[7]), tt = m_tan(s[7]);
        const T sc = T(1) / ct;
        f[6] = p + (sf * q + cf * r) * tt;
        f[7] = cf * q - sf * r;
        f[8] = (sf * q + cf * r) * sc;
        f[9] = (arm * (u[1] - u[3]) + q * r * (Jy - Jz)) / Jx;
        f[10] = (arm * (u[2] - u[0]) + p * r * (Jz - Jx)) / Jy;
        f[11] = (km * (u[0] - u[1] + u[2] - u[3]) + p * q * (Jx - Jy)) / Jz;
        if (fs) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                fs[i * NS + 3 + i] = T(1);
#pragma unroll
                for (int a = 0; a < 3; ++a) fs[(3 + i) * NS + 6 + a] = dR[a][i * 3 + 2] * thrust / mass;
            }
            const T w1 = sf * q + cf * r, w2 = cf * q - sf * r;
            fs[6 * NS + 6] = w2 * tt;
            fs[6 * NS + 7] = w1 * sc * sc;
            fs[6 * NS + 9] = T(1);
            fs[6 * NS + 10] = sf * tt;
            fs[6 * NS + 11] = cf * tt;
            fs[7 * NS + 6] = -w1;
            fs[7 * NS + 10] = cf;
            fs[7 * NS + 11] = -sf;
            fs[8 * NS + 6] = w2 * sc;
            fs[8 * NS + 7] = w1 * sc * tt;
            fs[8 * NS + 10] = sf * sc;
            fs[8 * NS + 11] = cf * sc;
            fs[9 * NS + 10] = r * (Jy - Jz) / Jx;
            fs[9 * NS + 11] = q * (Jy - Jz) / Jx;
            fs[10 * NS + 9] = r * (Jz - Jx) / Jy;
            fs[10 * NS + 11] = p * (Jz - Jx) / Jy;
            fs[11 * NS + 9] = q * (Jx - Jy) / Jz;
            fs[11 * NS + 10] = p * (Jx - Jy) / Jz;
        }
        if (fu) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) fu[(3 + i) * NU + k] = R[i * 3 + 2] / mass;
            fu[9 * NU + 1] = arm / Jx;
            fu[9 * NU + 3] = -arm / Jx;
            fu[10 * NU + 0] = -arm / Jy;
            fu[10 * NU + 2] = arm / Jy;
            fu[11 * NU + 0] = km / Jz;
            fu[11 * NU + 1] = -km / Jz;
            fu[11 * NU + 2] = km / Jz;
            fu[11 * NU + 3] = -km / Jz;
        }
    }
}

}  // namespace oca
