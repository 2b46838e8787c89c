// Host-side entry points that prepare the inputs of the hot path: the
// HEALPix ray set (Sec. 3.2) and the binned spectrum (Eq. gamma_shld with
// the cross sections of App. C1).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace urchin {
namespace {

// App. C1 cross sections, energies in eV.
double sigma_verner(double E)
{
    // Verner et al. (1996) H I fit, sigma_0 (x-1)^2 x^(P/2 - 11/2) (1 + sqrt(x/x_a))^(-P),
    // x = E/E_0, E_0 = 0.4298 eV, sigma_0 = 5.475e4 Mb, x_a = 32.88, P = 2.963
    if (E < kRydbergEV) return 0.0;
    const double x = E / 0.4298, P = 2.963;
    const double xm1 = x - 1.0;
    return 5.475e-14 * xm1 * xm1 * std::pow(x, 0.5 * P - 5.5) * std::pow(1.0 + std::sqrt(x / 32.88), -P);
}

double sigma_hydrogenic(double E, double Z = 1.0)
{
    // exact hydrogenic ion of charge Z (App. C1 for Z = 1; He II for Z = 2):
    // (sigma_th / Z^2) (nu_th/nu)^4 e^(4 - 4 atan(eps)/eps) / (1 - e^(-2 pi/eps)),
    // nu_th = Z^2 x 13.6 eV, eps = sqrt(nu/nu_th - 1); the bracket tends to 1 at threshold
    const double Eth = Z * Z * kRydbergEV;
    if (E < Eth) return 0.0;
    const double r = E / Eth;
    const double eps = std::sqrt(r - 1.0);
    double f = 1.0;
    if (eps > 1e-6) f = std::exp(4.0 - 4.0 * std::atan(eps) / eps) / (-std::expm1(-2.0 * kPi / eps));
    return sigma_th_cm2() / (Z * Z) * f / (r * r * r * r);
}

double sigma_powerlaw(double E)
{
    if (E < kRydbergEV) return 0.0;
    const double r = kRydbergEV / E;
    return sigma_th_cm2() * r * r * r;
}

}  // namespace
}  // namespace urchin

extern "C" int urchin_healpix_dirs(int nside, double* dirs_out)
{
    using namespace urchin;
    clear_error();
    if (nside < 1 || 12LL * nside * nside > URCHIN_MAX_RAYS)
        return set_error(URCHIN_ERR_ARG, "urchin_healpix_dirs: nside = %d out of range", nside);
    if (!dirs_out) return set_error(URCHIN_ERR_ARG, "urchin_healpix_dirs: dirs_out is NULL");
    // Ring scheme of Gorski et al. (2005): rings i = 1 .. 4 N_side - 1 from the
    // north pole; polar-cap rings hold 4i pixels at z = +-(1 - i^2/(3 N_side^2))
    // with azimuths 2 pi (j + 1/2)/(4i); equatorial rings (N_side <= i <= 3 N_side)
    // hold 4 N_side pixels at z = 4/3 - 2i/(3 N_side) with azimuths
    // 2 pi (j + 1 - s/2)/(4 N_side), s = (i - N_side + 1) mod 2; pixels are
    // numbered ring by ring in increasing azimuth.
    const double ns = (double)nside;
    int p = 0;
    for (int i = 1; i <= 4 * nside - 1; ++i) {
        double z;
        int npix;
        double shift;
        if (i < nside) {
            z = 1.0 - (double)i * i / (3.0 * ns * ns);
            npix = 4 * i;
            shift = 0.5;
        } else if (i <= 3 * nside) {
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns);
            npix = 4 * nside;
            shift = 1.0 - 0.5 * (double)((i - nside + 1) % 2);
        } else {
            int ii = 4 * nside - i;
            z = -(1.0 - (double)ii * ii / (3.0 * ns * ns));
            npix = 4 * ii;
            shift = 0.5;
        }
        const double st = std::sqrt(std::fmax(0.0, (1.0 - z) * (1.0 + z)));
        for (int j = 0; j < npix; ++j) {
            const double phi = 2.0 * kPi * ((double)j + shift) / (double)npix;
            dirs_out[3 * p] = st * std::cos(phi);
            dirs_out[3 * p + 1] = st * std::sin(phi);
            dirs_out[3 * p + 2] = z;
            ++p;
        }
    }
    return URCHIN_OK;
}

extern "C" int urchin_spectrum_weights(int F, const double* E_edges, const double* J, int xsec,
                                       double gamma_thin, double* s_out, double* w_out)
{
    using namespace urchin;
    clear_error();
    if (F < 1 || F > URCHIN_MAX_BINS) return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: F = %d", F);
    if (!E_edges || !J || !s_out || !w_out) return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: NULL array");
    if (xsec != URCHIN_XSEC_VERNER && xsec != URCHIN_XSEC_HYDROGENIC && xsec != URCHIN_XSEC_POWERLAW)
        return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: unknown cross section %d", xsec);
    if (!(gamma_thin > 0.0) || !std::isfinite(gamma_thin))
        return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: gamma_thin must be > 0");
    for (int j = 0; j <= F; ++j)
        if (!std::isfinite(E_edges[j]) || (j > 0 && !(E_edges[j] > E_edges[j - 1])))
            return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: edges must increase");
    if (E_edges[0] < kRydbergEV * (1.0 - 1e-3))
        return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: first edge below 13.6 eV");
    const double sth = sigma_th_cm2();
    double total = 0.0;
    for (int j = 0; j < F; ++j) {
        if (!std::isfinite(J[j]) || J[j] < 0.0) return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: bad J");
        const double Ec = std::sqrt(E_edges[j] * E_edges[j + 1]);   // geometric bin centre
        double sig = xsec == URCHIN_XSEC_HYDROGENIC ? sigma_hydrogenic(Ec)
                   : xsec == URCHIN_XSEC_POWERLAW   ? sigma_powerlaw(Ec)
                                                    : sigma_verner(Ec);
        s_out[j] = sig / sth;
        // Gamma = 4 pi int J sigma / (h nu) dnu: the bin contributes J sigma dE / E
        w_out[j] = J[j] * sig * (E_edges[j + 1] - E_edges[j]) / Ec;
        total += w_out[j];
    }
    if (!(total > 0.0)) return set_error(URCHIN_ERR_ARG, "urchin_spectrum_weights: zero total rate");
    const double scale = gamma_thin / total;
    for (int j = 0; j < F; ++j) w_out[j] *= scale;
    return URCHIN_OK;
}

extern "C" int urchin_cross_section_ratio(int F, const double* E_edges, int xsec, double* s_out)
{
    using namespace urchin;
    clear_error();
    if (F < 1 || F > URCHIN_MAX_BINS) return set_error(URCHIN_ERR_ARG, "urchin_cross_section_ratio: F = %d", F);
    if (!E_edges || !s_out) return set_error(URCHIN_ERR_ARG, "urchin_cross_section_ratio: NULL array");
    if (xsec != URCHIN_XSEC_VERNER && xsec != URCHIN_XSEC_HYDROGENIC && xsec != URCHIN_XSEC_POWERLAW &&
        xsec != URCHIN_XSEC_HEII)
        return set_error(URCHIN_ERR_ARG, "urchin_cross_section_ratio: unknown cross section %d", xsec);
    for (int j = 0; j <= F; ++j)
        if (!std::isfinite(E_edges[j]) || !(E_edges[j] > 0.0) || (j > 0 && !(E_edges[j] > E_edges[j - 1])))
            return set_error(URCHIN_ERR_ARG, "urchin_cross_section_ratio: edges must be positive and increase");
    const double sth = sigma_th_cm2();
    for (int j = 0; j < F; ++j) {
        const double Ec = std::sqrt(E_edges[j] * E_edges[j + 1]);
        const double sig = xsec == URCHIN_XSEC_HYDROGENIC ? sigma_hydrogenic(Ec)
                         : xsec == URCHIN_XSEC_HEII       ? sigma_hydrogenic(Ec, 2.0)
                         : xsec == URCHIN_XSEC_POWERLAW   ? sigma_powerlaw(Ec)
                                                          : sigma_verner(Ec);
        s_out[j] = sig / sth;
    }
    return URCHIN_OK;
}
