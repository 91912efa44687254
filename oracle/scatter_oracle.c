/*
 * scatter_oracle.c — plain FP64 CPU oracle for the direct kinematic
 * scattering sum (Favre-Nicolin et al., J. Appl. Cryst. 2010).
 *
 * TEST INFRASTRUCTURE.  This file is the definition the GPU library is
 * checked against.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Everything is written as the plain definition, in double precision, with a
 * straight loop over reflections (OpenMP-parallel) and atoms: no centring of
 * positions, no splitting of S, no blocking, no reordering.
 *
 * Conventions (readings of the paper, Sections 2.1 and 4):
 *   - positions r_j in lattice units, S in reciprocal lattice units, so that
 *     S.r_j is a phase in cycles; sign exp(+2 i pi S.r_j) (Eq. 2);
 *   - |S| in 1/Angstrom = |S_rlu| / a for the cubic reference lattice of
 *     parameter a; scattering-factor argument s = sin(theta)/lambda = |S|/2;
 *   - species coefficients are 12 doubles per species:
 *       a0 a1 a2 a3  b0 b1 b2 b3  c  f'  f''  B_dw
 *     f(s) = (sum_i a_i exp(-b_i s^2) + c + f' + i f'') * exp(-B_dw s^2)
 *     (analytic Gaussian-sum approximation of pynx.fthomson, Section 3;
 *      f', f'' and Debye-Waller factored per species, Section 4.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_NCOEF 12

static const double kPi = 3.14159265358979323846264338327950288;

/* Scattering factor of one species at |S| (1/Angstrom); Section 3
 * (pynx.fthomson Gaussian sum) and Section 4.2 (f', f'', Debye-Waller). */
void oracle_form_factor(const double* coef, double q_inv_angstrom, double* re, double* im) {
  const double s = 0.5 * q_inv_angstrom;
  const double s2 = s * s;
  double f0 = coef[8];
  for (int i = 0; i < 4; ++i) f0 += coef[i] * exp(-coef[4 + i] * s2);
  const double dw = exp(-coef[11] * s2);
  *re = (f0 + coef[9]) * dw;
  *im = coef[10] * dw;
}

/* |S| in 1/Angstrom for S in r.l.u. of a cubic lattice of parameter a. */
static double s_norm(const double* S, double lattice_a) {
  return sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]) / lattice_a;
}

/*
 * Eq. 2 for one reflection S, with occupancies (Section 3) and per-species
 * scattering factors (Section 4.2):
 *   A(S) = sum_j w_j f_{s(j)}(|S|) exp(2 i pi S.r_j).
 */
static void sum_one(int64_t n_atoms, const double* xyz, const int32_t* species,
                    const double* occ, const double* coef, double lattice_a,
                    const double* Sm, double* out) {
  const double q = s_norm(Sm, lattice_a);
  double are = 0.0, aim = 0.0;
  for (int64_t j = 0; j < n_atoms; ++j) {
    const double* r = xyz + 3 * j;
    const double phase = 2.0 * kPi * (Sm[0] * r[0] + Sm[1] * r[1] + Sm[2] * r[2]);
    const double c = cos(phase), s = sin(phase);
    const double w = occ ? occ[j] : 1.0;
    const int32_t sp = species ? species[j] : 0;
    double fr, fi;
    oracle_form_factor(coef + ORACLE_NCOEF * sp, q, &fr, &fi);
    /* w * f * (c + i s) */
    are += w * (fr * c - fi * s);
    aim += w * (fr * s + fi * c);
  }
  out[0] = are;
  out[1] = aim;
}

/*
 * A(S) of Eq. 2 for a list of reflections.
 *  xyz      [n_atoms][3]          species [n_atoms] (NULL: all 0)
 *  occ      [n_atoms] or NULL (all 1)
 *  coef     [n_species][12]       (n_species is implied by the indices)
 *  S        [n_s][3]              A out [n_s][2] (re, im)
 */
void oracle_amplitude(int64_t n_atoms, const double* xyz, const int32_t* species,
                      const double* occ, int32_t n_species, const double* coef,
                      double lattice_a, int64_t n_s, const double* S, double* A) {
  (void)n_species;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t m = 0; m < n_s; ++m)
    sum_one(n_atoms, xyz, species, occ, coef, lattice_a, S + 3 * m, A + 2 * m);
}

/*
 * Eq. 4: scattering from blocks of atoms (groups of unit cells), each block j
 * of type t(j) with its own structure factor F_t(S) at every reflection:
 *   A(S_m) = sum_j w_j F_{t(j)}(S_m) exp(2 i pi S_m.r_j),
 * r_j = r_j^0 + u_j the displaced block origin.  F is given as a table
 * [n_types][n_s][2] (re, im) of the caller's (for single-atom blocks it is
 * f_t(|S|), and the sum is Eq. 2).
 */
void oracle_amplitude_table(int64_t n_atoms, const double* xyz, const int32_t* types,
                            const double* occ, int32_t n_types, const double* table,
                            int64_t n_s, const double* S, double* A) {
  (void)n_types;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t m = 0; m < n_s; ++m) {
    const double* Sm = S + 3 * m;
    double are = 0.0, aim = 0.0;
    for (int64_t j = 0; j < n_atoms; ++j) {
      const double* r = xyz + 3 * j;
      const double phase = 2.0 * kPi * (Sm[0] * r[0] + Sm[1] * r[1] + Sm[2] * r[2]);
      const double c = cos(phase), s = sin(phase);
      const double w = occ ? occ[j] : 1.0;
      const int32_t t = types ? types[j] : 0;
      const double fr = table[2 * (t * n_s + m)], fi = table[2 * (t * n_s + m) + 1];
      are += w * (fr * c - fi * s);
      aim += w * (fr * s + fi * c);
    }
    A[2 * m] = are;
    A[2 * m + 1] = aim;
  }
}

/*
 * Eq. 5/6: the FFT approximation.  Every atom is put on the nearest node R_j
 * of a grid of step d (lattice units) from `origin`, r_j = R_j + u_j, and
 * the factor exp(2 i pi (S - H).u_j) is dropped, which is exact when
 * (S - H).u_j = 0 and a good approximation while |(S - H).u_j| << 1
 * (Eq. 7):
 *   A(S) ~ sum_j w_j f_{s(j)}(|S|) exp(2 i pi H.r_j) exp(2 i pi (S - H).R_j),
 * written here as that sum itself (no transform), for the reflections S.
 */
void oracle_fft_approx(int64_t n_atoms, const double* xyz, const int32_t* species,
                       const double* occ, int32_t n_species, const double* coef,
                       double lattice_a, const double* H, double step, const double* origin,
                       int64_t n_s, const double* S, double* A) {
  (void)n_species;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t m = 0; m < n_s; ++m) {
    const double* Sm = S + 3 * m;
    const double q = s_norm(Sm, lattice_a);
    double are = 0.0, aim = 0.0;
    for (int64_t j = 0; j < n_atoms; ++j) {
      const double* r = xyz + 3 * j;
      double R[3];
      for (int d = 0; d < 3; ++d) R[d] = origin[d] + step * nearbyint((r[d] - origin[d]) / step);
      const double phase = 2.0 * kPi * (H[0] * r[0] + H[1] * r[1] + H[2] * r[2] +
                                        (Sm[0] - H[0]) * R[0] + (Sm[1] - H[1]) * R[1] + (Sm[2] - H[2]) * R[2]);
      const double c = cos(phase), s = sin(phase);
      const double w = occ ? occ[j] : 1.0;
      const int32_t sp = species ? species[j] : 0;
      double fr, fi;
      oracle_form_factor(coef + ORACLE_NCOEF * sp, q, &fr, &fi);
      are += w * (fr * c - fi * s);
      aim += w * (fr * s + fi * c);
    }
    A[2 * m] = are;
    A[2 * m + 1] = aim;
  }
}

/*
 * Fresnel reflection and transmission coefficients of the substrate surface
 * (Section 3, pynx.gid; Section 4.3) for a wave in vacuum meeting a medium of
 * index n = 1 - delta + i beta at grazing angle alpha (rad):
 *   k_z  = sin(alpha)
 *   k_z' = sqrt(n^2 - cos^2(alpha))   (principal branch, Im >= 0:
 *                                      the field decays into the substrate)
 *   R = (k_z - k_z') / (k_z + k_z'),  T = 1 + R.
 */
/* sin of the refracted grazing angle in a medium of index n = 1 - delta + i beta:
 * q = sqrt(n^2 - cos^2 alpha), principal branch (Im q >= 0), so that k_z' = k q. */
static void refracted_sin(double alpha, double delta, double beta, double* q_re, double* q_im) {
  /* n^2 = (1 - delta)^2 - beta^2 + 2 i beta (1 - delta) */
  const double n2_re = (1.0 - delta) * (1.0 - delta) - beta * beta;
  const double n2_im = 2.0 * beta * (1.0 - delta);
  const double ca = cos(alpha);
  const double z_re = n2_re - ca * ca, z_im = n2_im;
  /* principal complex square root of z */
  const double mod = hypot(z_re, z_im);
  double k_re = sqrt(0.5 * (mod + z_re));
  double k_im = sqrt(fmax(0.0, 0.5 * (mod - z_re)));
  if (z_im < 0) k_im = -k_im;
  *q_re = k_re;
  *q_im = k_im;
}

void oracle_fresnel(double alpha, double delta, double beta, double* R, double* T) {
  const double kz = sin(alpha);
  double k_re, k_im;
  refracted_sin(alpha, delta, beta, &k_re, &k_im);
  /* R = (kz - k') / (kz + k') */
  const double nr = kz - k_re, ni = -k_im;
  const double dr = kz + k_re, di = k_im;
  const double den = dr * dr + di * di;
  R[0] = (nr * dr + ni * di) / den;
  R[1] = (ni * dr - nr * di) / den;
  T[0] = 1.0 + R[0];
  T[1] = R[1];
}

/*
 * Grazing-incidence amplitude in the distorted-wave Born approximation
 * (Section 4.3).  The paper names the four scattered beams (incident and exit
 * waves each either direct or reflected by the substrate) and the Fresnel
 * coefficients, but prints no formula; the reading used here is the island
 * in vacuum above a reflecting substrate, substrate scattering ignored:
 *
 *   A = sum_{t=1..4} W_t sum_j w_j f_{s(j)}(|S_t|) exp(2 i pi S_t.r_j)
 *   S_t = (h, k, Sz_t),  Sz in r.l.u. = a/lambda * (...)
 *     t=1: W=1        Sz = +(sin a_i + sin a_f)   (direct in, direct out)
 *     t=2: W=R_i      Sz = +(sin a_f - sin a_i)   (reflected in, direct out)
 *     t=3: W=R_f      Sz = -(sin a_f - sin a_i)   (direct in, reflected out)
 *     t=4: W=R_i R_f  Sz = -(sin a_i + sin a_f)   (reflected in and out)
 *   R_i = R(alpha_i), R_f = R(alpha_f) from oracle_fresnel.
 *
 *  pts  [n_pts][3] = (h, k, alpha_f in rad)     A out [n_pts][2]
 */
void oracle_dwba(int64_t n_atoms, const double* xyz, const int32_t* species,
                 const double* occ, int32_t n_species, const double* coef,
                 double lattice_a, double wavelength, double alpha_i, double delta,
                 double beta, int64_t n_pts, const double* pts, double* A) {
  (void)n_species;
  double Ri[2], Ti[2];
  oracle_fresnel(alpha_i, delta, beta, Ri, Ti);
  const double scale = lattice_a / wavelength;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t m = 0; m < n_pts; ++m) {
    const double h = pts[3 * m], k = pts[3 * m + 1], af = pts[3 * m + 2];
    double Rf[2], Tf[2];
    oracle_fresnel(af, delta, beta, Rf, Tf);
    const double sz[4] = {scale * (sin(alpha_i) + sin(af)), scale * (sin(af) - sin(alpha_i)),
                          -scale * (sin(af) - sin(alpha_i)), -scale * (sin(alpha_i) + sin(af))};
    double W[4][2];
    W[0][0] = 1.0;   W[0][1] = 0.0;
    W[1][0] = Ri[0]; W[1][1] = Ri[1];
    W[2][0] = Rf[0]; W[2][1] = Rf[1];
    W[3][0] = Ri[0] * Rf[0] - Ri[1] * Rf[1];
    W[3][1] = Ri[0] * Rf[1] + Ri[1] * Rf[0];
    double are = 0.0, aim = 0.0;
    for (int t = 0; t < 4; ++t) {
      const double St[3] = {h, k, sz[t]};
      double Tt[2];
      sum_one(n_atoms, xyz, species, occ, coef, lattice_a, St, Tt);
      are += W[t][0] * Tt[0] - W[t][1] * Tt[1];
      aim += W[t][0] * Tt[1] + W[t][1] * Tt[0];
    }
    A[2 * m] = are;
    A[2 * m + 1] = aim;
  }
}

/* g(S) = 4 (|A|^2 - I_obs) conj(A) at every reflection, and the misfit
 * L = sum_S (|A(S)|^2 - I_obs(S))^2 (serial sum in reflection order). */
static double misfit_and_g(int64_t n_s, const double* A, const double* I_obs, double* g) {
  double L = 0.0;
  for (int64_t m = 0; m < n_s; ++m) {
    const double I = A[2 * m] * A[2 * m] + A[2 * m + 1] * A[2 * m + 1];
    const double d = I - I_obs[m];
    L += d * d;
    g[2 * m] = 4.0 * d * A[2 * m];
    g[2 * m + 1] = -4.0 * d * A[2 * m + 1];
  }
  return L;
}

/* dL/dr_j of one atom:
 *   -2 pi sum_S S * Im( g(S) w_j f_{s(j)}(|S|) exp(2 i pi S.r_j) ). */
static void grad_one_atom(const double* r, double w, const double* coef_s, double lattice_a,
                          int64_t n_s, const double* S, const double* g, double* out) {
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int64_t m = 0; m < n_s; ++m) {
    const double* Sm = S + 3 * m;
    double fr, fi;
    oracle_form_factor(coef_s, s_norm(Sm, lattice_a), &fr, &fi);
    const double phase = 2.0 * kPi * (Sm[0] * r[0] + Sm[1] * r[1] + Sm[2] * r[2]);
    const double c = cos(phase), s = sin(phase);
    /* e = w f (c + i s);  Im(g e) */
    const double er = w * (fr * c - fi * s), ei = w * (fr * s + fi * c);
    const double im_ge = g[2 * m] * ei + g[2 * m + 1] * er;
    gx += Sm[0] * im_ge;
    gy += Sm[1] * im_ge;
    gz += Sm[2] * im_ge;
  }
  out[0] = -2.0 * kPi * gx;
  out[1] = -2.0 * kPi * gy;
  out[2] = -2.0 * kPi * gz;
}

/*
 * Grazing incidence on an object buried in the substrate (the reading of the
 * buried case of Section 4.3, where the paper names the transmission
 * coefficients beside the reflection ones and prints no formula): the
 * substrate fills z < 0 below a flat surface at z = 0 (lattice units), the
 * atoms lie inside it (z <= 0), and the substrate has no lower interface, so
 * inside it there is one incident wave, transmitted with T_i = T(alpha_i), and
 * one wave towards the detector, transmitted with T_f = T(alpha_f).  Both are
 * refracted: with q = sqrt(n^2 - cos^2 alpha) (Im q >= 0) the in-medium
 * momentum transfer along z is (a / lambda)(q_i + q_f), and both waves decay
 * with depth, e^{(2 pi a / lambda)(Im q_i + Im q_f) z} for z <= 0.  So
 *   A(h, k, alpha_f) = T_i T_f sum_s f_s(|S_1|) sum_{j in s} w_j
 *                        exp(2 i pi (h x_j + k y_j + sigma z_j)),
 *   sigma = (a / lambda)(conj(q_i) + conj(q_f)),
 * with f at the vacuum beam S_1 = (h, k, (a / lambda)(sin a_i + sin a_f)).
 * With delta = beta = 0, T = 1 and sigma = S_1z: the kinematic sum at S_1.
 *
 *  pts  [n_pts][3] = (h, k, alpha_f in rad)     A out [n_pts][2]
 */
void oracle_dwba_buried(int64_t n_atoms, const double* xyz, const int32_t* species,
                        const double* occ, int32_t n_species, const double* coef,
                        double lattice_a, double wavelength, double alpha_i, double delta,
                        double beta, int64_t n_pts, const double* pts, double* A) {
  (void)n_species;
  double Ri[2], Ti[2], qi_re, qi_im;
  oracle_fresnel(alpha_i, delta, beta, Ri, Ti);
  refracted_sin(alpha_i, delta, beta, &qi_re, &qi_im);
  const double scale = lattice_a / wavelength;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t m = 0; m < n_pts; ++m) {
    const double h = pts[3 * m], k = pts[3 * m + 1], af = pts[3 * m + 2];
    double Rf[2], Tf[2], qf_re, qf_im;
    oracle_fresnel(af, delta, beta, Rf, Tf);
    refracted_sin(af, delta, beta, &qf_re, &qf_im);
    const double sig_re = scale * (qi_re + qf_re), sig_im = -scale * (qi_im + qf_im);
    const double S1[3] = {h, k, scale * (sin(alpha_i) + sin(af))};
    const double q = s_norm(S1, lattice_a);
    double are = 0.0, aim = 0.0;
    for (int64_t j = 0; j < n_atoms; ++j) {
      const double* r = xyz + 3 * j;
      const double phase = 2.0 * kPi * (h * r[0] + k * r[1] + sig_re * r[2]);
      const double damp = exp(-2.0 * kPi * sig_im * r[2]);
      const double c = damp * cos(phase), s = damp * sin(phase);
      const double w = occ ? occ[j] : 1.0;
      double fr, fi;
      oracle_form_factor(coef + ORACLE_NCOEF * (species ? species[j] : 0), q, &fr, &fi);
      are += w * (fr * c - fi * s);
      aim += w * (fr * s + fi * c);
    }
    /* T_i T_f times the sum */
    const double tr = Ti[0] * Tf[0] - Ti[1] * Tf[1], ti = Ti[0] * Tf[1] + Ti[1] * Tf[0];
    A[2 * m] = tr * are - ti * aim;
    A[2 * m + 1] = tr * aim + ti * are;
  }
}

/*
 * Misfit of an intensity map and its analytic gradient (adjoint of Eq. 2):
 *   L = sum_S (|A(S)|^2 - I_obs(S))^2
 *   dL/dr_j = -2 pi sum_S S * Im( g(S) w_j f_{s(j)}(|S|) exp(2 i pi S.r_j) ),
 *   g(S) = 4 (|A(S)|^2 - I_obs(S)) conj(A(S)),
 * with f held fixed as a function of S.  A is recomputed here by
 * oracle_amplitude.  grad out [n_atoms][3] (may be NULL), *loss out.
 */
void oracle_loss_grad(int64_t n_atoms, const double* xyz, const int32_t* species,
                      const double* occ, int32_t n_species, const double* coef,
                      double lattice_a, int64_t n_s, const double* S, const double* I_obs,
                      double* loss, double* grad) {
  double* A = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  double* g = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  oracle_amplitude(n_atoms, xyz, species, occ, n_species, coef, lattice_a, n_s, S, A);
  *loss = misfit_and_g(n_s, A, I_obs, g);
  if (grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_atoms; ++j)
      grad_one_atom(xyz + 3 * j, occ ? occ[j] : 1.0, coef + ORACLE_NCOEF * (species ? species[j] : 0),
                    lattice_a, n_s, S, g, grad + 3 * j);
  }
  free(A);
  free(g);
}

/*
 * Misfit and analytic gradient of Eq. 4 (blocks with per-(type, S) factors
 * F_t(S) from a table [n_types][n_s][2], block origins r_j = r_j^0 + u_j),
 * F held fixed:
 *   dL/dr_j = -2 pi sum_S S * Im( g(S) w_j F_{t(j)}(S) exp(2 i pi S.r_j) ),
 *   g(S) = 4 (|A(S)|^2 - I_obs(S)) conj(A(S)),  A from oracle_amplitude_table.
 * grad out [n_atoms][3] (may be NULL), *loss out.
 */
void oracle_loss_grad_table(int64_t n_atoms, const double* xyz, const int32_t* types,
                            const double* occ, int32_t n_types, const double* table,
                            int64_t n_s, const double* S, const double* I_obs,
                            double* loss, double* grad) {
  double* A = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  double* g = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  oracle_amplitude_table(n_atoms, xyz, types, occ, n_types, table, n_s, S, A);
  *loss = misfit_and_g(n_s, A, I_obs, g);
  if (grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_atoms; ++j) {
      const double* r = xyz + 3 * j;
      const double w = occ ? occ[j] : 1.0;
      const int32_t t = types ? types[j] : 0;
      double gx = 0.0, gy = 0.0, gz = 0.0;
      for (int64_t m = 0; m < n_s; ++m) {
        const double* Sm = S + 3 * m;
        const double fr = table[2 * (t * n_s + m)], fi = table[2 * (t * n_s + m) + 1];
        const double phase = 2.0 * kPi * (Sm[0] * r[0] + Sm[1] * r[1] + Sm[2] * r[2]);
        const double c = cos(phase), s = sin(phase);
        /* e = w F (c + i s);  Im(g e) */
        const double er = w * (fr * c - fi * s), ei = w * (fr * s + fi * c);
        const double im_ge = g[2 * m] * ei + g[2 * m + 1] * er;
        gx += Sm[0] * im_ge;
        gy += Sm[1] * im_ge;
        gz += Sm[2] * im_ge;
      }
      grad[3 * j] = -2.0 * kPi * gx;
      grad[3 * j + 1] = -2.0 * kPi * gy;
      grad[3 * j + 2] = -2.0 * kPi * gz;
    }
  }
  free(A);
  free(g);
}

/*
 * The same misfit and analytic gradient, for the selected atoms only and from
 * an amplitude map A [n_s][2] the caller already has (oracle_amplitude's
 * output): for maps too large to sum more than once.
 *  atoms [n_sel] indices; grad out [n_sel][3] (may be NULL), *loss out.
 */
void oracle_loss_grad_given_amplitude(int64_t n_atoms, const double* xyz, const int32_t* species,
                                      const double* occ, int32_t n_species, const double* coef,
                                      double lattice_a, int64_t n_s, const double* S, const double* A,
                                      const double* I_obs, int64_t n_sel, const int64_t* atoms,
                                      double* loss, double* grad) {
  (void)n_atoms;
  (void)n_species;
  double* g = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  *loss = misfit_and_g(n_s, A, I_obs, g);
  if (grad) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_sel; ++q) {
      const int64_t j = atoms[q];
      grad_one_atom(xyz + 3 * j, occ ? occ[j] : 1.0, coef + ORACLE_NCOEF * (species ? species[j] : 0),
                    lattice_a, n_s, S, g, grad + 3 * q);
    }
  }
  free(g);
}

/*
 * Central finite differences of L for selected atoms, a route to the
 * gradient independent of the adjoint formula.  Moving atom j by +-h along
 * axis d changes only its own term of Eq. 2, so
 *   A+-(S) = A(S) + w_j f (exp(2 i pi S.(r_j +- h e_d)) - exp(2 i pi S.r_j))
 * and, with I+- = |A+-|^2, the difference of the two misfits is taken as
 *   L+ - L- = sum_S (I+ - I-) (I+ + I- - 2 I_obs)
 * (difference of squares: no cancellation between two large sums).
 *   grad_d = (L+ - L-) / (2 h).
 * A [n_s][2] is the unperturbed map (oracle_amplitude's output).
 *
 *  atoms [n_sel] indices; grad out [n_sel][3].
 */
void oracle_fd_grad_given_amplitude(int64_t n_atoms, const double* xyz, const int32_t* species,
                                    const double* occ, int32_t n_species, const double* coef,
                                    double lattice_a, int64_t n_s, const double* S, const double* A,
                                    const double* I_obs, int64_t n_sel, const int64_t* atoms, double h,
                                    double* grad) {
  (void)n_atoms;
  (void)n_species;
  for (int64_t q = 0; q < n_sel; ++q) {
    const int64_t j = atoms[q];
    const double* r = xyz + 3 * j;
    const double w = occ ? occ[j] : 1.0;
    const int32_t sp = species ? species[j] : 0;
    for (int d = 0; d < 3; ++d) {
      double diff = 0.0;
#pragma omp parallel for reduction(+ : diff) schedule(static)
      for (int64_t m = 0; m < n_s; ++m) {
        const double* Sm = S + 3 * m;
        double fr, fi;
        oracle_form_factor(coef + ORACLE_NCOEF * sp, s_norm(Sm, lattice_a), &fr, &fi);
        const double p0 = 2.0 * kPi * (Sm[0] * r[0] + Sm[1] * r[1] + Sm[2] * r[2]);
        const double pp = p0 + 2.0 * kPi * Sm[d] * h;
        const double pm = p0 - 2.0 * kPi * Sm[d] * h;
        /* e(p) = w f (cos p + i sin p) */
        const double c0 = cos(p0), s0 = sin(p0);
        const double cp = cos(pp), sp_ = sin(pp);
        const double cm = cos(pm), sm = sin(pm);
        /* d+- = A+- - A */
        const double dpr = w * (fr * (cp - c0) - fi * (sp_ - s0));
        const double dpi = w * (fr * (sp_ - s0) + fi * (cp - c0));
        const double dmr = w * (fr * (cm - c0) - fi * (sm - s0));
        const double dmi = w * (fr * (sm - s0) + fi * (cm - c0));
        /* I+ - I- = Re((A+ - A-) conj(A+ + A-)), A+ - A- taken directly */
        const double ddr = w * (fr * (cp - cm) - fi * (sp_ - sm));
        const double ddi = w * (fr * (sp_ - sm) + fi * (cp - cm));
        const double sr = 2.0 * A[2 * m] + dpr + dmr, si = 2.0 * A[2 * m + 1] + dpi + dmi;
        const double dI = ddr * sr + ddi * si;
        const double apr = A[2 * m] + dpr, api = A[2 * m + 1] + dpi;
        const double amr = A[2 * m] + dmr, ami = A[2 * m + 1] + dmi;
        const double Ip = apr * apr + api * api, Im = amr * amr + ami * ami;
        diff += dI * (Ip + Im - 2.0 * I_obs[m]);
      }
      grad[3 * q + d] = diff / (2.0 * h);
    }
  }
}

/* oracle_fd_grad_given_amplitude with A computed here by oracle_amplitude. */
void oracle_fd_grad(int64_t n_atoms, const double* xyz, const int32_t* species,
                    const double* occ, int32_t n_species, const double* coef,
                    double lattice_a, int64_t n_s, const double* S, const double* I_obs,
                    int64_t n_sel, const int64_t* atoms, double h, double* grad) {
  double* A = (double*)malloc(sizeof(double) * 2 * (size_t)n_s);
  oracle_amplitude(n_atoms, xyz, species, occ, n_species, coef, lattice_a, n_s, S, A);
  oracle_fd_grad_given_amplitude(n_atoms, xyz, species, occ, n_species, coef, lattice_a, n_s, S, A, I_obs,
                                 n_sel, atoms, h, grad);
  free(A);
}

/* Threads of the following calls (timing the oracle on one core); n < 1
 * restores the runtime default.  Host control only: no effect on results. */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  static int default_n = 0;
  if (default_n == 0) default_n = omp_get_max_threads();
  omp_set_num_threads(n >= 1 ? n : default_n);
#else
  (void)n;
#endif
}

/* Number of OpenMP threads the oracle runs with (for reporting). */
int oracle_num_threads(void) {
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    {
#ifdef _OPENMP
      n = omp_get_num_threads();
#endif
    }
  }
  return n;
}
