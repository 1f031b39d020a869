// Far-image operator of the periodic evaluation (Sec. 2.4: periodic boundary
// conditions; the Coulomb lattice sum exists only for a neutral cell).
//
// The periodic KIFMM takes the cell (side L, half-width h = L / 2) as the
// root and runs its lists over the cell and its 26 neighbouring images.  All
// farther images act on the root through one matrix: T[j][k] is the
// potential, in the units of Eq. 3 (kernel 1 / (4 pi r)), at the root's
// downward check point y_j = 1.05 h S_j of a unit charge at its upward
// equivalent point z_k = 1.05 h S_k repeated over every image cell n with
// max |n_i| >= 2.  That sum converges only conditionally, so it is taken as
// Ewald's sum of the unit charge (split parameter a = 3 / L; real-space
// images up to 5 cells away, reciprocal vectors k = 2 pi m / L up to the
// shell where exp(-k^2 / 4 a^2) < 1e-17; no k = 0 term, i.e. a uniform
// neutralising background, which cancels on a neutral density) minus its 27
// nearest images.  Each near image is subtracted inside the real-space term,
// erfc(a r) / r - 1 / r = -erf(a r) / r, so the difference stays finite where
// the two surfaces meet (the limit -2 a / sqrt(pi) at r = 0).
//
// Host code in FP64, run once per plan (cell and surface order fixed).
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace kifmm {

cudaError_t far_image_operator(int p, double L, double *T) {
    const std::vector<double> S = unit_surface(p);
    const int n = (int)(S.size() / 3);
    const double h = 0.5 * L, rad = kAlphaInner * h;  // DC and UE radii are both 1.05 h
    const double a = 3.0 / L;
    const double pi = 3.14159265358979323846;
    const int shells = 5;
    std::vector<double> acc((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
            const double r0[3] = {rad * (S[3 * j] - S[3 * k]), rad * (S[3 * j + 1] - S[3 * k + 1]),
                                  rad * (S[3 * j + 2] - S[3 * k + 2])};
            double sum = 0.0;
            for (int ix = -shells; ix <= shells; ++ix)
                for (int iy = -shells; iy <= shells; ++iy)
                    for (int iz = -shells; iz <= shells; ++iz) {
                        const double dx = r0[0] + L * ix, dy = r0[1] + L * iy, dz = r0[2] + L * iz;
                        const double d = std::sqrt(dx * dx + dy * dy + dz * dz);
                        const bool near = std::abs(ix) <= 1 && std::abs(iy) <= 1 && std::abs(iz) <= 1;
                        if (near)
                            sum += (d > 0.0) ? -std::erf(a * d) / d : -2.0 * a / std::sqrt(pi);
                        else
                            sum += std::erfc(a * d) / d;
                    }
            acc[(size_t)j * n + k] = sum;
        }
    // reciprocal space: cos(k.(y - z)) = cos(k.y) cos(k.z) + sin(k.y) sin(k.z)
    const int kmax = (int)std::ceil(a * L * std::sqrt(4.0 * 39.2) / (2.0 * pi));
    std::vector<double> cy(n), sy(n), cz(n), sz(n);
    for (int mx = -kmax; mx <= kmax; ++mx)
        for (int my = -kmax; my <= kmax; ++my)
            for (int mz = -kmax; mz <= kmax; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                const double kx = 2.0 * pi / L * mx, ky = 2.0 * pi / L * my, kz = 2.0 * pi / L * mz;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double w = 4.0 * pi / (L * L * L) * std::exp(-k2 / (4.0 * a * a)) / k2;
                for (int j = 0; j < n; ++j) {
                    const double ph = rad * (kx * S[3 * j] + ky * S[3 * j + 1] + kz * S[3 * j + 2]);
                    cy[j] = std::cos(ph);
                    sy[j] = std::sin(ph);
                }
                for (int j = 0; j < n; ++j)
                    for (int k = 0; k < n; ++k)
                        acc[(size_t)j * n + k] += w * (cy[j] * cy[k] + sy[j] * sy[k]);
            }
    for (size_t i = 0; i < acc.size(); ++i) T[i] = acc[i] / (4.0 * pi);
    return cudaSuccess;
}

}  // namespace kifmm

using namespace kifmm;

kifmm_status kifmm_far_image_operator(int p, double cell, double *T) {
    if (p < 2 || p > 10 || !T || !(cell > 0.0) || !std::isfinite(cell)) return KIFMM_ERR_ARG;
    return far_image_operator(p, cell, T) == cudaSuccess ? KIFMM_OK : KIFMM_ERR_CUDA;
}
