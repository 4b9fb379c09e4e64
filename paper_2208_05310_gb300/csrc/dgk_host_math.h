// dgk_host_math.h -- host-side set-up math of libdgk (operators, saturation states).
#pragma once

#include <string>
#include <vector>

namespace dgk {
namespace host {

struct Operators1D {
    int P;
    double xi[16], w[16];
    double D[256], Dhat[256];
    double lm[16], lp[16];  // l_j(-1), l_j(+1)
    // mortars: Im[h][j*P+i] = l_i((xi_j + 2h - 1)/2), the basis of a face at the points of
    // its half h (h = 0 lower, 1 upper)
    double Im[2][256];
};

bool gauss_legendre(int n, double *x, double *w);
bool dg_operators(int N, Operators1D &op);
double pressure(double rho, double T);
bool maxwell(double T, double &rho_v, double &rho_l);
bool sigma_vl(double T, double gammaK, double &sigma);

// Curved elements (dgk_geom.cpp): node coordinates x [D][ne][NP], metric terms
// met [D*D+1][ne][NP] (plane i*D + k: J a^i_k; plane D*D: 1/J) and face metrics
// fmet [D][ne][NF][NFP] (J a^dir_k at the points of face f = 2 dir + side).
struct CurvedGeometry {
    std::vector<double> met, fmet, x;
};
// conn: unstructured connectivity [ne][NF][3] (neighbour or -1 - wall, its face, face-point
// orientation) or null for the box's; the tables are checked against the element maps.
bool curved_geometry(int D, const Operators1D &op, int ngeo, const int n[3], const int periodic[3], long long ne,
                     const double *xgeo, const int *conn, CurvedGeometry &out, std::string &err);

}  // namespace host
}  // namespace dgk
