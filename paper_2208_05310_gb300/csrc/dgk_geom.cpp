// dgk_geom.cpp -- host set-up of curved elements (Sec. 3.1, curvilinear elements): node
// coordinates and metric terms of polynomial element maps, in double.
//
// Element e maps the reference cube [-1,1]^D by the tensor-product polynomial of degree
// ngeo per direction through the caller's points at t_a = -1 + 2a/ngeo.  At the
// Legendre-Gauss nodes and at the face points the map is evaluated by sum factorisation
// (one 1D operator per direction: the Lagrange basis of the t_a or its derivative), and
// the metric terms are the cofactors of the Jacobian matrix dX/dxi:
//   J a^i = dX/dxi_{i+1} x dX/dxi_{i+2} (cyclic; in 2D the rotated columns), J = det.
// They are polynomials of degree <= 2 ngeo (3D; ngeo in 2D) per direction, which the
// Gauss collocation differentiates exactly when 2 ngeo <= N (ngeo <= N): then the
// discrete metric identities hold and a uniform state is preserved.  The face metric of
// a face shared by two elements is computed once, from the element on the face's minus
// side, and used by both (one normal and surface element per face point: conservation).
// With unstructured connectivity tables the face's owner is the element with the smaller
// index, and the tables are checked against the element maps (the other element's own
// face metric must agree with the owner's after the face-point orientation).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dgk_host_math.h"

namespace dgk {
namespace host {

namespace {

// l_a(x) and l_a'(x) of the equispaced points t_0..t_g
void lagrange_equispaced(int g, double x, double *l, double *dl)
{
    double t[17];
    for (int a = 0; a <= g; ++a) t[a] = -1.0 + 2.0 * a / g;
    for (int a = 0; a <= g; ++a) {
        double den = 1.0, val = 1.0;
        for (int k = 0; k <= g; ++k)
            if (k != a) {
                den *= t[a] - t[k];
                val *= x - t[k];
            }
        double der = 0.0;
        for (int m = 0; m <= g; ++m) {
            if (m == a) continue;
            double prod = 1.0;
            for (int k = 0; k <= g; ++k)
                if (k != a && k != m) prod *= x - t[k];
            der += prod;
        }
        l[a] = val / den;
        dl[a] = der / den;
    }
}

// out[i0 + n0 (i1 + n1 i2)] = sum_abc B0[i0][a] B1[i1][b] B2[i2][c] in[a + G (b + G c)]
// (D = 2: B2 and the third index absent); Bd is n_d x G, row-major.
void tensor_apply(int D, int G, const double *B0, int n0, const double *B1, int n1, const double *B2, int n2,
                  const double *in, double *out, std::vector<double> &w1, std::vector<double> &w2)
{
    const int G2 = D == 3 ? G : 1, m2 = D == 3 ? n2 : 1;
    w1.assign((size_t)n0 * G * G2, 0.0);
    for (int c = 0; c < G2; ++c)
        for (int b = 0; b < G; ++b)
            for (int i0 = 0; i0 < n0; ++i0) {
                double s = 0.0;
                for (int a = 0; a < G; ++a) s += B0[i0 * G + a] * in[a + G * (b + G * c)];
                w1[i0 + n0 * (b + G * c)] = s;
            }
    w2.assign((size_t)n0 * n1 * G2, 0.0);
    for (int c = 0; c < G2; ++c)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i0 = 0; i0 < n0; ++i0) {
                double s = 0.0;
                for (int b = 0; b < G; ++b) s += B1[i1 * G + b] * w1[i0 + n0 * (b + G * c)];
                w2[i0 + n0 * (i1 + n1 * c)] = s;
            }
    if (D == 2) {
        for (int i = 0; i < n0 * n1; ++i) out[i] = w2[i];
        return;
    }
    for (int i2 = 0; i2 < m2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i0 = 0; i0 < n0; ++i0) {
                double s = 0.0;
                for (int c = 0; c < G; ++c) s += B2[i2 * G + c] * w2[i0 + n0 * (i1 + n1 * c)];
                out[i0 + n0 * (i1 + n1 * i2)] = s;
            }
}

// cofactors: Ja[i][k] = (J a^i)_k from J[j][k] = d X_k / d xi_j; returns det
double cofactors(int D, const double J[3][3], double Ja[3][3])
{
    if (D == 2) {
        Ja[0][0] = J[1][1];
        Ja[0][1] = -J[1][0];
        Ja[1][0] = -J[0][1];
        Ja[1][1] = J[0][0];
        return J[0][0] * J[1][1] - J[0][1] * J[1][0];
    }
    for (int i = 0; i < 3; ++i) {
        const int p = (i + 1) % 3, q = (i + 2) % 3;
        for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            Ja[i][k] = J[p][k1] * J[q][k2] - J[p][k2] * J[q][k1];
        }
    }
    return J[0][0] * Ja[0][0] + J[0][1] * Ja[0][1] + J[0][2] * Ja[0][2];
}

}  // namespace

bool curved_geometry(int D, const Operators1D &op, int ngeo, const int n[3], const int periodic[3], long long ne,
                     const double *xgeo, const int *conn, CurvedGeometry &out, std::string &err)
{
    const int P = op.P, G = ngeo + 1;
    const int NP = D == 2 ? P * P : P * P * P, NFP = D == 2 ? P : P * P, NF = 2 * D;
    const int NG = D == 2 ? G * G : G * G * G;
    if (ngeo < 1 || ngeo > 16) {
        err = "ngeo must be 1..16";
        return false;
    }
    // 1D operators: values and derivatives at the nodes (P x G) and at xi = -1, +1 (1 x G)
    std::vector<double> L(P * G), dL(P * G), Le[2], dLe[2];
    for (int i = 0; i < P; ++i) lagrange_equispaced(ngeo, op.xi[i], &L[i * G], &dL[i * G]);
    for (int s = 0; s < 2; ++s) {
        Le[s].resize(G);
        dLe[s].resize(G);
        lagrange_equispaced(ngeo, s ? 1.0 : -1.0, Le[s].data(), dLe[s].data());
    }
    out.met.assign((size_t)(D * D + 1) * ne * NP, 0.0);
    out.fmet.assign((size_t)D * ne * NF * NFP, 0.0);
    out.x.assign((size_t)D * ne * NP, 0.0);
    std::vector<double> w1, w2, Xe(NG);
    // values / derivatives of all coordinates at a set of points (the nodes, or one face)
    std::vector<double> pv[3], pd[3][3];
    for (long long e = 0; e < ne; ++e) {
        auto eval = [&](int face_dir, int side, int npts) {
            for (int k = 0; k < D; ++k) {
                for (int g = 0; g < NG; ++g) Xe[g] = xgeo[((size_t)k * ne + e) * NG + g];
                pv[k].resize(npts);
                const double *B[3] = {nullptr, nullptr, nullptr}, *Bd[3] = {nullptr, nullptr, nullptr};
                int nn[3] = {1, 1, 1};
                for (int d = 0; d < D; ++d) {
                    const bool f = d == face_dir;
                    B[d] = f ? Le[side].data() : L.data();
                    Bd[d] = f ? dLe[side].data() : dL.data();
                    nn[d] = f ? 1 : P;
                }
                tensor_apply(D, G, B[0], nn[0], B[1], nn[1], B[2], nn[2], Xe.data(), pv[k].data(), w1, w2);
                for (int j = 0; j < D; ++j) {
                    pd[j][k].resize(npts);
                    const double *C[3] = {B[0], B[1], B[2]};
                    C[j] = Bd[j];
                    tensor_apply(D, G, C[0], nn[0], C[1], nn[1], C[2], nn[2], Xe.data(), pd[j][k].data(), w1, w2);
                }
            }
        };
        eval(-1, 0, NP);
        for (int p = 0; p < NP; ++p) {
            double Jm[3][3] = {{0}}, Ja[3][3] = {{0}};
            for (int j = 0; j < D; ++j)
                for (int k = 0; k < D; ++k) Jm[j][k] = pd[j][k][p];
            const double det = cofactors(D, Jm, Ja);
            if (!(det > 0.0) || !std::isfinite(det)) {
                err = "an element map is not orientation-preserving (J <= 0 at a node)";
                return false;
            }
            for (int i = 0; i < D; ++i)
                for (int k = 0; k < D; ++k) out.met[((size_t)(i * D + k) * ne + e) * NP + p] = Ja[i][k];
            out.met[((size_t)(D * D) * ne + e) * NP + p] = 1.0 / det;
            for (int k = 0; k < D; ++k) out.x[((size_t)k * ne + e) * NP + p] = pv[k][p];
        }
        for (int f = 0; f < NF; ++f) {
            const int dir = f / 2, side = f % 2;
            eval(dir, side, NFP);
            for (int p = 0; p < NFP; ++p) {
                double Jm[3][3] = {{0}}, Ja[3][3] = {{0}};
                for (int j = 0; j < D; ++j)
                    for (int k = 0; k < D; ++k) Jm[j][k] = pd[j][k][p];
                cofactors(D, Jm, Ja);
                for (int k = 0; k < D; ++k) out.fmet[(((size_t)k * ne + e) * NF + f) * NFP + p] = Ja[dir][k];
            }
        }
    }
    if (conn) {
        // unstructured: a shared face takes the metric of the element with the smaller
        // index (of the smaller face for an element facing itself), mapped to the other
        // element's face points and frame (opposite outward normals: J a^dir = nsign *
        // outward).  The other element's own metric must agree: a check that the tables
        // match the element maps.
        for (long long e = 0; e < ne; ++e)
            for (int f = 0; f < NF; ++f) {
                const int *c = conn + (e * NF + f) * 3;
                const long long nb = c[0];
                const int fo = c[1], o = c[2];
                // walls and both sides of mortars keep their own face metrics
                if (nb < 0 || (o >> 3) || nb < e || (nb == e && fo < f)) continue;
                const double sg = ((f ^ fo) & 1) ? 1.0 : -1.0;
                for (int p = 0; p < NFP; ++p) {
                    const int a = p % P, b = p / P;
                    int u = (o & 1) ? b : a, v = (o & 1) ? a : b;
                    if (o & 2) u = P - 1 - u;
                    if (o & 4) v = P - 1 - v;
                    const int q = u + P * v;
                    double diff = 0.0, mag = 0.0;
                    for (int k = 0; k < D; ++k) {
                        const double own = out.fmet[(((size_t)k * ne + e) * NF + f) * NFP + p];
                        double &dst = out.fmet[(((size_t)k * ne + nb) * NF + fo) * NFP + q];
                        diff += (dst - sg * own) * (dst - sg * own);
                        mag += own * own;
                        dst = sg * own;
                    }
                    if (diff > 1e-12 * mag) {
                        err = "the connectivity does not match the element maps (element " + std::to_string(e) + ", face " +
                              std::to_string(f) + ")";
                        return false;
                    }
                }
            }
        return true;
    }
    // minus faces with a neighbour take the neighbour's plus-face metric
    const long long stride[3] = {1, n[0], (long long)n[0] * n[1]};
    for (long long e = 0; e < ne; ++e) {
        const long long co[3] = {e % n[0], (e / n[0]) % n[1], D == 3 ? e / ((long long)n[0] * n[1]) : 0};
        for (int dir = 0; dir < D; ++dir) {
            long long b;
            if (co[dir] > 0) b = e - stride[dir];
            else if (periodic[dir]) b = e + (long long)(n[dir] - 1) * stride[dir];
            else continue;
            for (int k = 0; k < D; ++k)
                std::memcpy(&out.fmet[(((size_t)k * ne + e) * NF + 2 * dir) * NFP],
                            &out.fmet[(((size_t)k * ne + b) * NF + 2 * dir + 1) * NFP], NFP * sizeof(double));
        }
    }
    return true;
}

}  // namespace host
}  // namespace dgk
