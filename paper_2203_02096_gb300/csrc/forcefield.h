// forcefield.h -- the library's force-field constants.
//
// The paper names the interaction terms (Section II-A: van der Waals,
// hydrogen bonding, electrostatics, desolvation, particle-grid interaction)
// but prints no functional form or constant.  The forms used here: 12-6
// Lennard-Jones with minimum -eps_ij at R_ij = (R_i+R_j)/2, eps_ij =
// sqrt(eps_i eps_j); 12-10 hydrogen bond between a donor (HD) and an
// acceptor (NA, OA, SA) with minimum -eps_hb at R_hb of the acceptor;
// screened Coulomb with the sigmoidal dielectric of Mehler and Solmajer
// (1991); Gaussian desolvation (S_i V_j + S_j V_i) exp(-r^2 / 2 sigma^2),
// S = solpar + q_solv |q|.  Every pair term is evaluated at max(r, 0.5 A);
// intramolecular pairs are cut at 8 A.  All constants are this library's
// own choices.
#pragma once

namespace ff {

struct AtomType {
    double R, eps, vol, solpar;
    int hb;          // 0 none, 1 donor, 2 acceptor
    double Rhb, ehb; // acceptor's 12-10 minimum and depth
};

// C, A, N, NA, OA, SA, HD
static const AtomType kTypes[7] = {
    {4.0, 0.15, 33.5, -0.0015, 0, 0.0, 0.0},  {4.0, 0.15, 33.5, -0.0005, 0, 0.0, 0.0},
    {3.5, 0.16, 22.5, -0.0015, 0, 0.0, 0.0},  {3.5, 0.16, 22.5, -0.0015, 2, 1.9, 5.0},
    {3.2, 0.20, 17.0, -0.0025, 2, 1.9, 5.0},  {4.0, 0.20, 33.5, -0.0020, 2, 2.5, 1.0},
    {2.0, 0.02, 0.0, 0.0005, 1, 0.0, 0.0},
};

constexpr double kWvdw = 0.16, kWhb = 0.12, kWel = 0.14, kWds = 0.13;
constexpr double kQsolv = 0.011;
constexpr double kCoulomb = 332.06;
constexpr double kDielA = -8.5525, kDielEps0 = 78.4, kDielLambda = 0.003627, kDielK = 7.7839;
constexpr double kDielB = kDielEps0 - kDielA;
constexpr double kSigma = 3.6;
constexpr double kCutoff = 8.0;
constexpr double kRFloor = 0.5;
constexpr double kKout = 10.0;
constexpr double kMapCap = 1.0e5;

inline bool hbond_pair(int a, int b) {
    return (kTypes[a].hb == 1 && kTypes[b].hb == 2) || (kTypes[a].hb == 2 && kTypes[b].hb == 1);
}

// Pair coefficients of E = c12/r^12 - c6/r^6 - c10/r^10 (weights folded in).
inline void vdw_coefs(int a, int b, double &c12, double &c6, double &c10) {
    if (hbond_pair(a, b)) {
        const AtomType &acc = kTypes[a].hb == 2 ? kTypes[a] : kTypes[b];
        double r2 = acc.Rhb * acc.Rhb, r10 = r2 * r2 * r2 * r2 * r2;
        c12 = kWhb * 5.0 * acc.ehb * r10 * r2;
        c10 = kWhb * 6.0 * acc.ehb * r10;
        c6 = 0.0;
    } else {
        double R = 0.5 * (kTypes[a].R + kTypes[b].R), e = __builtin_sqrt(kTypes[a].eps * kTypes[b].eps);
        double r6 = R * R * R * R * R * R;
        c12 = kWvdw * e * r6 * r6;
        c6 = kWvdw * 2.0 * e * r6;
        c10 = 0.0;
    }
}

inline double solv(int t, double q) { return kTypes[t].solpar + kQsolv * (q < 0 ? -q : q); }

}  // namespace ff
