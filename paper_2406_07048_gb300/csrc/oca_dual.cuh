// Forward-mode dual numbers v + d*eps (eps^2 = 0) for the adjoint kernels.
//
// The model and pose templates (oca_models.cuh) and the stage assembly
// (oca_stage.cuh) are written once over a number type T.  Instantiated with
// Dual<T> and one input's tangent set to 1, they return that input's
// partial derivatives alongside the values, which is how the backward pass
// gets the second derivatives of the dynamics and of the part poses that
// the linearisation point of each trajectory step depends on.
#pragma once

#include "oca_common.cuh"

namespace oca {

template <typename T>
struct Dual {
    T v, d;
    OCA_HD Dual() : v(T(0)), d(T(0)) {}
    OCA_HD Dual(T x) : v(x), d(T(0)) {}
    OCA_HD Dual(T x, T dx) : v(x), d(dx) {}
    OCA_HD Dual &operator+=(const Dual &o) { v += o.v; d += o.d; return *this; }
    OCA_HD Dual &operator-=(const Dual &o) { v -= o.v; d -= o.d; return *this; }
    OCA_HD Dual &operator*=(const Dual &o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
    OCA_HD Dual &operator/=(const Dual &o) { const T q = v / o.v; d = (d - q * o.d) / o.v; v = q; return *this; }
};

template <typename T> OCA_HD inline Dual<T> operator+(Dual<T> a, const Dual<T> &b) { return a += b; }
template <typename T> OCA_HD inline Dual<T> operator-(Dual<T> a, const Dual<T> &b) { return a -= b; }
template <typename T> OCA_HD inline Dual<T> operator*(Dual<T> a, const Dual<T> &b) { return a *= b; }
template <typename T> OCA_HD inline Dual<T> operator/(Dual<T> a, const Dual<T> &b) { return a /= b; }
template <typename T> OCA_HD inline Dual<T> operator-(const Dual<T> &a) { return Dual<T>(-a.v, -a.d); }
// mixed forms with the underlying scalar
template <typename T> OCA_HD inline Dual<T> operator+(Dual<T> a, T b) { a.v += b; return a; }
template <typename T> OCA_HD inline Dual<T> operator+(T b, Dual<T> a) { a.v += b; return a; }
template <typename T> OCA_HD inline Dual<T> operator-(Dual<T> a, T b) { a.v -= b; return a; }
template <typename T> OCA_HD inline Dual<T> operator-(T b, const Dual<T> &a) { return Dual<T>(b - a.v, -a.d); }
template <typename T> OCA_HD inline Dual<T> operator*(Dual<T> a, T b) { a.v *= b; a.d *= b; return a; }
template <typename T> OCA_HD inline Dual<T> operator*(T b, Dual<T> a) { a.v *= b; a.d *= b; return a; }
template <typename T> OCA_HD inline Dual<T> operator/(Dual<T> a, T b) { a.v /= b; a.d /= b; return a; }
template <typename T> OCA_HD inline Dual<T> operator/(T b, const Dual<T> &a) {
    const T q = b / a.v;
    return Dual<T>(q, -q * a.d / a.v);
}

// elementary functions: value and chain-rule tangent
template <typename T> OCA_HD inline Dual<T> m_sin(const Dual<T> &a) { return Dual<T>(m_sin(a.v), m_cos(a.v) * a.d); }
template <typename T> OCA_HD inline Dual<T> m_cos(const Dual<T> &a) { return Dual<T>(m_cos(a.v), -m_sin(a.v) * a.d); }
template <typename T> OCA_HD inline Dual<T> m_tan(const Dual<T> &a) {
    const T t = m_tan(a.v);
    return Dual<T>(t, (T(1) + t * t) * a.d);
}
template <typename T> OCA_HD inline Dual<T> m_sqrt(const Dual<T> &a) {
    const T r = m_sqrt(a.v);
    return Dual<T>(r, a.d / (T(2) * r));
}

// the model with every parameter a constant (zero tangent)
template <typename T>
OCA_HD inline DevModel<Dual<T>> dual_model(const DevModel<T> &m) {
    DevModel<Dual<T>> o;
    o.kind = m.kind;
    o.dt = Dual<T>(m.dt);
    for (int i = 0; i < 8; ++i) o.p[i] = Dual<T>(m.p[i]);
    for (int i = 0; i < 12; ++i) {
        o.Qs[i] = Dual<T>(m.Qs[i]);
        o.s_lo[i] = Dual<T>(m.s_lo[i]);
        o.s_hi[i] = Dual<T>(m.s_hi[i]);
    }
    for (int i = 0; i < 4; ++i) {
        o.Qu[i] = Dual<T>(m.Qu[i]);
        o.u_lo[i] = Dual<T>(m.u_lo[i]);
        o.u_hi[i] = Dual<T>(m.u_hi[i]);
    }
    return o;
}

}  // namespace oca
