// dgk_host_math.h -- host-side set-up math of libdgk (operators, saturation states).
#pragma once

namespace dgk {
namespace host {

struct Operators1D {
    int P;
    double xi[16], w[16];
    double D[256], Dhat[256];
    double lm[16], lp[16];  // l_j(-1), l_j(+1)
};

bool gauss_legendre(int n, double *x, double *w);
bool dg_operators(int N, Operators1D &op);
double pressure(double rho, double T);
bool maxwell(double T, double &rho_v, double &rho_l);
bool sigma_vl(double T, double gammaK, double &sigma);

}  // namespace host
}  // namespace dgk
