// Host-side check of the device lens math (compiled by nvcc as host code):
// the per-system-constant EPL deflection against the generic series, and its
// analytic vector-Jacobian product against forward-mode dual numbers and
// central differences.  Prints the worst relative errors.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include "rtu_math.cuh"

using namespace rtu;

static double urand(unsigned& s) { s = s * 1664525u + 1013904223u; return (s >> 8) / 16777216.0; }

int main() {
    unsigned seed = 12345u;
    double worst_val = 0, worst_dual = 0, worst_fd = 0;
    for (int trial = 0; trial < 400; ++trial) {
        const bool epl = trial % 3 != 0;
        double q = 0.55 + 0.4 * urand(seed), phi = 3.14159 * urand(seed);
        double c = (1 - q) / (1 + q);
        double p[6] = {0.8 + urand(seed), 1.7 + 0.6 * urand(seed), c * cos(2 * phi), c * sin(2 * phi),
                       0.2 * (urand(seed) - 0.5), 0.2 * (urand(seed) - 0.5)};
        double x = 4 * (urand(seed) - 0.5), y = 4 * (urand(seed) - 0.5);
        double gx = urand(seed) - 0.5, gy = urand(seed) - 0.5;
        EplC<double> C;
        epl_setup(C, p, epl, 1e-17);
        double ax, ay;
        epl_alpha(C, x, y, ax, ay);
        // generic series (the oracle's formulation)
        double bx, by;
        epl_deflect<double>(x, y, p[0], epl ? p[1] : 2.0, p[2], p[3], p[4], p[5], bx, by, 1e-17, 400);
        // relative error of the deflection vector (a component can be near zero)
        worst_val = fmax(worst_val, sqrt((ax - bx) * (ax - bx) + (ay - by) * (ay - by)) /
                                        fmax(1e-12, sqrt(bx * bx + by * by)));
        // analytic VJP
        double out[6] = {0, 0, 0, 0, 0, 0}, vx, vy;
        epl_alpha_vjp(C, epl, x, y, gx, gy, vx, vy, out);
        // forward-mode duals
        typedef Dual<double, 6> D;
        D dx_, dy_;
        epl_deflect<D>(D(x), D(y), D::seed(p[0], 0), epl ? D::seed(p[1], 1) : D(2.0), D::seed(p[2], 2),
                       D::seed(p[3], 3), D::seed(p[4], 4), D::seed(p[5], 5), dx_, dy_, 1e-17, 400);
        double nrm = 0, err = 0, efd = 0;
        for (int k = 0; k < 6; ++k) {
            if (!epl && k == 1) continue;
            double ref = gx * dx_.d[k] + gy * dy_.d[k];
            nrm += ref * ref;
            err += (out[k] - ref) * (out[k] - ref);
            // central difference of the value path
            double pp[6], pm[6];
            for (int j = 0; j < 6; ++j) { pp[j] = p[j]; pm[j] = p[j]; }
            const double h = 1e-6;
            pp[k] += h; pm[k] -= h;
            EplC<double> Cp, Cm;
            epl_setup(Cp, pp, epl, 1e-17);
            epl_setup(Cm, pm, epl, 1e-17);
            double a1, a2, b1, b2;
            epl_alpha(Cp, x, y, a1, b1);
            epl_alpha(Cm, x, y, a2, b2);
            double fd = (gx * (a1 - a2) + gy * (b1 - b2)) / (2 * h);
            efd += (out[k] - fd) * (out[k] - fd);
        }
        worst_dual = fmax(worst_dual, sqrt(err / fmax(nrm, 1e-300)));
        worst_fd = fmax(worst_fd, sqrt(efd / fmax(nrm, 1e-300)));
    }
    // the series tail bound: |alpha - alpha after m terms| <= epl_tail_bound
    double worst_tail = 0;
    for (int trial = 0; trial < 4000; ++trial) {
        const bool epl = trial % 3 != 0;
        double q = 0.3 + 0.69 * urand(seed), phi = 3.14159 * urand(seed);
        double c = (1 - q) / (1 + q);
        double p[6] = {0.5 + urand(seed), 1.2 + 1.6 * urand(seed), c * cos(2 * phi), c * sin(2 * phi),
                       0.2 * (urand(seed) - 0.5), 0.2 * (urand(seed) - 0.5)};
        double x = 6 * (urand(seed) - 0.5), y = 6 * (urand(seed) - 0.5);
        EplC<double> C;
        epl_setup(C, p, epl, 1e-17);
        double ax, ay;
        epl_alpha(C, x, y, ax, ay);
        for (int m = 0; m <= 4; ++m) {
            EplPart<double> ps;
            epl_alpha_begin(C, x, y, m, ps);
            double bx, by;
            epl_alpha_of(C, ps, bx, by);
            const double d = sqrt((ax - bx) * (ax - bx) + (ay - by) * (ay - by));
            const double bound = epl_tail_bound(C, ps);
            if (bound > 0) worst_tail = fmax(worst_tail, d / bound);
            else worst_tail = fmax(worst_tail, d > 1e-15 ? 1e9 : 0.0);
            double fx, fy;
            epl_alpha_finish(C, ps, fx, fy);
            if (fx != ax || fy != ay) worst_tail = 1e9;      // split sum must equal the plain sum
        }
    }
    printf("value %.3e dual %.3e fd %.3e tail %.3e\n", worst_val, worst_dual, worst_fd, worst_tail);
    return 0;
}
