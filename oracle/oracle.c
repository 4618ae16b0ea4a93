/*
 * oracle.c -- plain, slow FP64 CPU oracle for the capacitance -> Bz forward map of
 * capacitively tuned loop arrays and for its gradient.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load this library. The CUDA product path never calls it, and the
 * two share no code: this file includes no header of the CUDA library and vice versa.
 *
 * What it computes (paper: "Differentiable Cosimulator for Electrically Reconfigurable
 * Structures", Mueller, Philipp, Guenther):
 *   - Sec. I-A: for structures small against the wavelength the forward map C -> B is the
 *     circuit model combined with the Biot-Savart law. The field basis H[p][k] is the Bz
 *     at point p produced by 1 A in loop k (Biot-Savart, straight segments).
 *   - Eq. 2 and Eq. 11: each port is a loop closed by a capacitor; its impedance is
 *     R + j w L - j/(w C). Eq. 12-13: L + M, the self and mutual inductances, form the
 *     reactive coupling. The loop currents solve (R + j w M + diag(1/(j w C))) I = V.
 *   - Eq. 7: the field is the superposition B = H I of the per-port fields.
 *   - Eq. 1: the objective is the mean squared error against a target |Bz| (Sec. IV-C
 *     optimises |Hz| at collocation points).
 *   - Eq. 8-9: the derivative of the wave (current) vector follows from
 *     d(A^-1) = -A^-1 dA A^-1; both the direct (one solve per capacitor) and the
 *     adjoint (one solve per system) forms are written out here.
 *   - Eq. 3-7 and Eq. 10: the scattering-parameter route, used as an independent
 *     cross-check of the impedance route.
 *
 * Conventions: SI units, time dependence e^{+j w t} (Eq. 2, Eq. 11), mu0 = 4 pi 1e-7 H/m.
 * Matrices are dense row-major. Complex values are C99 double complex.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp]. Contraction of
 * a*b+c into a fused multiply-add is switched off so that x86 and Arm hosts produce
 * identical bits.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846
#define ORACLE_MU0 (4.0e-7 * ORACLE_PI)

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------
 * Biot-Savart field of one straight segment (Sec. I-A).
 *
 * Segment r1 -> r2 carrying 1 A, field point p. With R1 = r1 - p, R2 = r2 - p the
 * integral of mu0/(4 pi) dl x (p - l)/|p - l|^3 along the segment is
 *     B = mu0/(4 pi) (R1 x R2) (|R1| + |R2|) / (|R1| |R2| (|R1| |R2| + R1.R2)).
 * When R1.R2 < 0 (point beside the span) the sum |R1||R2| + R1.R2 cancels; the identity
 * (|R1||R2|)^2 - (R1.R2)^2 = |R1 x R2|^2 rewrites it as |R1 x R2|^2 / (|R1||R2| - R1.R2).
 * Inside the wire (perpendicular distance rho < wire radius rw, foot of the perpendicular
 * on the span) the field of a uniform current density grows linearly with rho, so the
 * term is scaled by rho^2 / rw^2 relative to the thin-wire expression (which is
 * proportional to 1/rho there). The paper does not treat this case; it is our reading.
 * Returns component `comp` (0: z, 1: x, 2: y) of the field; the direction of every
 * component is that of R1 x R2.
 * ------------------------------------------------------------------------------------ */
double oracle_segment_b(double x1, double y1, double z1, double x2, double y2, double z2,
                        double px, double py, double pz, double rw, int comp) {
  double R1[3] = {x1 - px, y1 - py, z1 - pz};
  double R2[3] = {x2 - px, y2 - py, z2 - pz};
  double d[3] = {x2 - x1, y2 - y1, z2 - z1};
  double c[3] = {R1[1] * R2[2] - R1[2] * R2[1], R1[2] * R2[0] - R1[0] * R2[2],
                 R1[0] * R2[1] - R1[1] * R2[0]};
  double n1 = sqrt(R1[0] * R1[0] + R1[1] * R1[1] + R1[2] * R1[2]);
  double n2 = sqrt(R2[0] * R2[0] + R2[1] * R2[1] + R2[2] * R2[2]);
  double dot = R1[0] * R2[0] + R1[1] * R2[1] + R1[2] * R2[2];
  double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
  double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (dd == 0.0) return 0.0; /* degenerate segment carries no field */
  /* perpendicular distance to the line and position of the foot along the span */
  double rho2 = c2 / dd; /* |R1 x d|^2/|d|^2 and R1 x d = R1 x R2 */
  double t = -(R1[0] * d[0] + R1[1] * d[1] + R1[2] * d[2]) / dd;
  double scale = 1.0;
  if (t >= 0.0 && t <= 1.0 && rho2 < rw * rw) {
    if (rho2 == 0.0) return 0.0; /* on the wire axis: field of a uniform current is 0 */
    scale = rho2 / (rw * rw);
  }
  double denom; /* |R1||R2| (|R1||R2| + R1.R2) */
  double f;
  if (dot >= 0.0) {
    denom = n1 * n2 * (n1 * n2 + dot);
    if (denom == 0.0) return 0.0; /* point on an endpoint */
    f = (n1 + n2) / denom;
  } else {
    if (c2 == 0.0) return 0.0;
    f = (n1 + n2) * (n1 * n2 - dot) / (n1 * n2 * c2);
  }
  const double cc = comp == 1 ? c[0] : (comp == 2 ? c[1] : c[2]);
  return ORACLE_MU0 / (4.0 * ORACLE_PI) * cc * f * scale;
}

/* The z component (the normal field Bz the configurations optimise). */
double oracle_segment_bz(double x1, double y1, double z1, double x2, double y2, double z2,
                         double px, double py, double pz, double rw) {
  return oracle_segment_b(x1, y1, z1, x2, y2, z2, px, py, pz, rw, 0);
}

/* Field basis H[p][k] (Sec. I-A; the per-port field of Eq. 7 at unit current): the sum
 * over the closed polyline of loop k (vertices loop_vtx_off[k] .. loop_vtx_off[k+1]-1,
 * last vertex joined back to the first) of oracle_segment_b, for the component comp[p]
 * of point p (0: z, 1: x, 2: y; comp NULL: z everywhere; Eq. 7 superposes all three). */
void oracle_basis_comp(int32_t n_loops, const int32_t* loop_vtx_off, const double* vx,
                       const double* vy, const double* vz, int64_t n_points, const double* px,
                       const double* py, const double* pz, const int8_t* comp, double rw,
                       double* H) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n_points; ++p) {
    for (int32_t k = 0; k < n_loops; ++k) {
      int32_t a = loop_vtx_off[k], b = loop_vtx_off[k + 1];
      double s = 0.0;
      for (int32_t v = a; v < b; ++v) {
        int32_t w = (v + 1 < b) ? v + 1 : a;
        s += oracle_segment_b(vx[v], vy[v], vz[v], vx[w], vy[w], vz[w], px[p], py[p], pz[p],
                              rw, comp ? comp[p] : 0);
      }
      H[p * n_loops + k] = s;
    }
  }
}

void oracle_basis(int32_t n_loops, const int32_t* loop_vtx_off, const double* vx,
                  const double* vy, const double* vz, int64_t n_points, const double* px,
                  const double* py, const double* pz, double rw, double* H) {
  oracle_basis_comp(n_loops, loop_vtx_off, vx, vy, vz, n_points, px, py, pz, NULL, rw, H);
}

/* ------------------------------------------------------------------------------------
 * Partial inductances of straight filaments (Eq. 12-13 use L + M; the paper extracts
 * them from the full-wave admittance, here they come from the Neumann integral
 * M = mu0/(4 pi) sum_ij int int dl_i . dl_j / |r_i - r_j| over segment pairs).
 *
 * Perpendicular segments: dl_i . dl_j = 0, so the term is 0.
 * Parallel segments at perpendicular offset d > 0 with axial spans [a1,a2], [b1,b2]:
 *   M = s mu0/(4 pi) [G(a2-b1) - G(a1-b1) - G(a2-b2) + G(a1-b2)],
 *   G(u) = u asinh(u/d) - sqrt(u^2 + d^2), s = +1 (same direction) or -1 (opposite).
 * Collinear segments (d = 0) that do not overlap: the d -> 0 limit of G is
 * |u| ln(2|u|/d) - |u| (u asinh(u/d) tends to |u| ln(2|u|/d)); the ln(2/d) parts cancel
 * between the four terms for non-overlapping spans, leaving G0(u) = |u| ln|u| - |u|
 * (0 ln 0 = 0).
 * A segment with itself: mu0 l/(2 pi) (ln(2 l / rw) - 1), the thin round wire without
 * internal inductance (skin depth far below the wire radius at these frequencies).
 * Pairs that are neither parallel nor perpendicular (oblique) and do not touch use the
 * Neumann integral by quadrature (oracle_segment_pair_quadrature).
 * Oblique pairs that share an end point O (the corners of a non-rectilinear polygon), with
 * far end points P and Q, lengths l = |OP|, m = |OQ| and R = |PQ|: the Neumann double
 * integral int_0^l int_0^m ds dt / |r1 - r2| of two rays from O at angle e, whose distance
 * is sqrt(s^2 + t^2 - 2 s t cos e), integrates in closed form to
 *   F = 2 [l atanh(m / (l + R)) + m atanh(l / (m + R))],
 * so M = mu0/(4 pi) (u1.u2) F with u1, u2 the current directions (oracle_touching_pair).
 * Status: 0 ok, 2 overlapping collinear segments.
 * ------------------------------------------------------------------------------------ */
static double oracle_G(double u, double d) { return u * asinh(u / d) - sqrt(u * u + d * d); }
static double oracle_G0(double u) {
  double a = fabs(u);
  return (a == 0.0) ? 0.0 : a * log(a) - a;
}

/* Gauss-Legendre rule of order n on [-1, 1]: the nodes are the roots of the Legendre
 * polynomial P_n (Newton's method from the Chebyshev-like guesses cos(pi (i + 3/4)/(n + 1/2)),
 * P_n and P_n' by the three-term recurrence), the weights 2 / ((1 - x^2) P_n'(x)^2). */
void oracle_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(ORACLE_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Integral of 1/|p - b(t)| along the straight segment b0 -> b1 (length l2, unit vector u2):
 * with w = p - b0, t0 = w.u2, rho^2 = |w|^2 - t0^2, it is
 *   asinh((l2 - t0)/rho) + asinh(t0/rho) = ln((R1 + l2 - t0) / (R0 - t0)),
 * R0 = |p - b0|, R1 = |p - b1|; a factor that cancels is rewritten through
 * (R - t)(R + t) = rho^2 (rho^2 itself cancels when the projection of p falls outside the
 * span). */
static double oracle_inv_distance_line(const double p[3], const double b0[3], const double u2[3],
                                       double l2) {
  double w0[3] = {p[0] - b0[0], p[1] - b0[1], p[2] - b0[2]};
  double t0 = w0[0] * u2[0] + w0[1] * u2[1] + w0[2] * u2[2];
  double R0 = sqrt(w0[0] * w0[0] + w0[1] * w0[1] + w0[2] * w0[2]);
  double w1[3] = {w0[0] - l2 * u2[0], w0[1] - l2 * u2[1], w0[2] - l2 * u2[2]};
  double R1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
  double a = l2 - t0;
  if (t0 <= 0.0) return log((R1 + a) / (R0 - t0)); /* projection before b0: no cancellation */
  if (a < 0.0) return log((R0 + t0) / (R1 - a));   /* beyond b1: both factors rewritten */
  double rho2 = R0 * R0 - t0 * t0;                   /* projection on the span */
  return log((R1 + a) * (R0 + t0) / rho2);
}

/* Distance from point p to the segment a -> b. */
static double oracle_point_segment_distance(const double p[3], const double a[3],
                                            const double b[3]) {
  double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double t = dd > 0.0 ? (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]) / dd : 0.0;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  double e[3] = {w[0] - t * d[0], w[1] - t * d[1], w[2] - t * d[2]};
  return sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
}

/* Panels of the outer rule: the outer segment is split into m equal panels with
 * m = min(8, ceil(l1 / d)), d the smallest distance from an end point of either segment to
 * the other segment, so that each panel is no longer than the gap (for segments that cross
 * without touching this d can overstate the gap). */
int oracle_quadrature_panels(const double r1s[3], const double r1e[3], const double r2s[3],
                             const double r2e[3]) {
  double l1 = sqrt((r1e[0] - r1s[0]) * (r1e[0] - r1s[0]) + (r1e[1] - r1s[1]) * (r1e[1] - r1s[1]) +
                   (r1e[2] - r1s[2]) * (r1e[2] - r1s[2]));
  double d = oracle_point_segment_distance(r1s, r2s, r2e);
  double t = oracle_point_segment_distance(r1e, r2s, r2e);
  if (t < d) d = t;
  t = oracle_point_segment_distance(r2s, r1s, r1e);
  if (t < d) d = t;
  t = oracle_point_segment_distance(r2e, r1s, r1e);
  if (t < d) d = t;
  if (!(d > 0.0)) return 8;
  double m = ceil(l1 / d);
  return m < 1.0 ? 1 : (m > 8.0 ? 8 : (int)m);
}

/* Mutual partial inductance of two straight filaments in any relative position that do not
 * touch: M = mu0/(4 pi) (u1.u2) int_0^l1 int_0^l2 ds dt / |r1(s) - r2(t)| (Neumann), the
 * inner integral in closed form and the outer one by the composite Gauss-Legendre rule of
 * the given order on oracle_quadrature_panels equal panels. */
double oracle_segment_pair_quadrature(const double r1s[3], const double r1e[3],
                                      const double r2s[3], const double r2e[3], int order) {
  double d1[3] = {r1e[0] - r1s[0], r1e[1] - r1s[1], r1e[2] - r1s[2]};
  double d2[3] = {r2e[0] - r2s[0], r2e[1] - r2s[1], r2e[2] - r2s[2]};
  double l1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
  double l2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
  if (l1 == 0.0 || l2 == 0.0) return 0.0;
  double u2[3] = {d2[0] / l2, d2[1] / l2, d2[2] / l2};
  double cosang = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (l1 * l2);
  double x[64], w[64];
  if (order > 64) order = 64;
  oracle_gauss_legendre(order, x, w);
  const int m = oracle_quadrature_panels(r1s, r1e, r2s, r2e);
  double acc = 0.0;
  for (int q = 0; q < m; ++q)
    for (int i = 0; i < order; ++i) {
      double s = (q + 0.5 * (x[i] + 1.0)) / m;
      double p[3] = {r1s[0] + s * d1[0], r1s[1] + s * d1[1], r1s[2] + s * d1[2]};
      acc += w[i] * oracle_inv_distance_line(p, r2s, u2, l2);
    }
  return ORACLE_MU0 / (4.0 * ORACLE_PI) * cosang * 0.5 * (l1 / m) * acc;
}

/* Neumann integral of two straight filaments that share the end point O (see the block
 * comment above): far end points P (of the first) and Q (of the second). Returns
 * mu0/(4 pi) cosang F, cosang the cosine between the two current directions. */
double oracle_touching_pair(const double O[3], const double P[3], const double Q[3],
                            double cosang) {
  double l = sqrt((P[0] - O[0]) * (P[0] - O[0]) + (P[1] - O[1]) * (P[1] - O[1]) +
                  (P[2] - O[2]) * (P[2] - O[2]));
  double m = sqrt((Q[0] - O[0]) * (Q[0] - O[0]) + (Q[1] - O[1]) * (Q[1] - O[1]) +
                  (Q[2] - O[2]) * (Q[2] - O[2]));
  double R = sqrt((P[0] - Q[0]) * (P[0] - Q[0]) + (P[1] - Q[1]) * (P[1] - Q[1]) +
                  (P[2] - Q[2]) * (P[2] - Q[2]));
  double F = 2.0 * (l * atanh(m / (l + R)) + m * atanh(l / (m + R)));
  return ORACLE_MU0 / (4.0 * ORACLE_PI) * cosang * F;
}

/* Order of the rule for oblique pairs (enough for segments farther apart than a tenth of
 * their length; pairs that touch take oracle_touching_pair). */
#define ORACLE_OBLIQUE_ORDER 16

static double oracle_dist2(const double a[3], const double b[3]) {
  double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return d0 * d0 + d1 * d1 + d2 * d2;
}

int oracle_segment_pair_inductance(const double r1s[3], const double r1e[3],
                                   const double r2s[3], const double r2e[3], double rw,
                                   int same_segment, double* out) {
  double d1[3] = {r1e[0] - r1s[0], r1e[1] - r1s[1], r1e[2] - r1s[2]};
  double d2[3] = {r2e[0] - r2s[0], r2e[1] - r2s[1], r2e[2] - r2s[2]};
  double l1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
  double l2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
  *out = 0.0;
  if (l1 == 0.0 || l2 == 0.0) return 0;
  if (same_segment) {
    *out = ORACLE_MU0 * l1 / (2.0 * ORACLE_PI) * (log(2.0 * l1 / rw) - 1.0);
    return 0;
  }
  double dot = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  double cx = d1[1] * d2[2] - d1[2] * d2[1];
  double cy = d1[2] * d2[0] - d1[0] * d2[2];
  double cz = d1[0] * d2[1] - d1[1] * d2[0];
  double cross = sqrt(cx * cx + cy * cy + cz * cz);
  double tol = 1e-12 * l1 * l2;
  if (fabs(dot) <= tol) return 0; /* perpendicular */
  if (cross > tol) {              /* oblique: quadrature unless the segments touch */
    double e2 = 1e-24 * (l1 + l2) * (l1 + l2);
    double cosang = dot / (l1 * l2);
    if (oracle_dist2(r1s, r2s) <= e2)
      *out = oracle_touching_pair(r1s, r1e, r2e, cosang);
    else if (oracle_dist2(r1s, r2e) <= e2)
      *out = oracle_touching_pair(r1s, r1e, r2s, cosang);
    else if (oracle_dist2(r1e, r2s) <= e2)
      *out = oracle_touching_pair(r1e, r1s, r2e, cosang);
    else if (oracle_dist2(r1e, r2e) <= e2)
      *out = oracle_touching_pair(r1e, r1s, r2s, cosang);
    else
      *out = oracle_segment_pair_quadrature(r1s, r1e, r2s, r2e, ORACLE_OBLIQUE_ORDER);
    return 0;
  }
  double u[3] = {d1[0] / l1, d1[1] / l1, d1[2] / l1};
  double w[3] = {r2s[0] - r1s[0], r2s[1] - r1s[1], r2s[2] - r1s[2]};
  double b_s = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
  double we[3] = {r2e[0] - r1s[0], r2e[1] - r1s[1], r2e[2] - r1s[2]};
  double b_e = we[0] * u[0] + we[1] * u[1] + we[2] * u[2];
  double perp[3] = {w[0] - b_s * u[0], w[1] - b_s * u[1], w[2] - b_s * u[2]};
  double dist = sqrt(perp[0] * perp[0] + perp[1] * perp[1] + perp[2] * perp[2]);
  double sgn = (dot > 0.0) ? 1.0 : -1.0;
  double a1 = 0.0, a2 = l1;
  double b1 = (b_s < b_e) ? b_s : b_e;
  double b2 = (b_s < b_e) ? b_e : b_s;
  double v;
  if (dist <= 1e-12 * (l1 + l2)) {
    /* overlapping collinear filaments diverge; spans that meet within rounding of their
     * lengths (consecutive pieces of one straight side) are the touching case of G0 */
    double ov = 1e-12 * (l1 + l2);
    if (b1 < a2 - ov && a1 < b2 - ov) return 2;
    v = oracle_G0(a2 - b1) - oracle_G0(a1 - b1) - oracle_G0(a2 - b2) + oracle_G0(a1 - b2);
  } else {
    v = oracle_G(a2 - b1, dist) - oracle_G(a1 - b1, dist) - oracle_G(a2 - b2, dist) +
        oracle_G(a1 - b2, dist);
  }
  *out = sgn * ORACLE_MU0 / (4.0 * ORACLE_PI) * v;
  return 0;
}

/* Inductance matrix M[k][l] = sum over segment pairs of loops k and l (Eq. 12: L on the
 * diagonal, mutual M off it). If L_self is not NULL, its entries replace the diagonal
 * (the closed-form loop inductance of a circular loop, for instance). Rows are independent
 * (threads over k; every entry is summed in the same order whatever the thread count).
 * Returns the largest pair status met (0 when every pair was handled). */
int oracle_inductance(int32_t n_loops, const int32_t* loop_vtx_off, const double* vx,
                      const double* vy, const double* vz, double rw, const double* L_self,
                      double* M) {
  int status = 0;
#pragma omp parallel for schedule(dynamic) reduction(max : status)
  for (int32_t k = 0; k < n_loops; ++k) {
    for (int32_t l = 0; l < n_loops; ++l) {
      if (k == l && L_self != NULL) {
        M[k * n_loops + l] = L_self[k];
        continue;
      }
      double s = 0.0;
      for (int32_t i = loop_vtx_off[k]; i < loop_vtx_off[k + 1]; ++i) {
        int32_t ie = (i + 1 < loop_vtx_off[k + 1]) ? i + 1 : loop_vtx_off[k];
        double a0[3] = {vx[i], vy[i], vz[i]}, a1[3] = {vx[ie], vy[ie], vz[ie]};
        for (int32_t j = loop_vtx_off[l]; j < loop_vtx_off[l + 1]; ++j) {
          int32_t je = (j + 1 < loop_vtx_off[l + 1]) ? j + 1 : loop_vtx_off[l];
          double b0[3] = {vx[j], vy[j], vz[j]}, b1[3] = {vx[je], vy[je], vz[je]};
          double m;
          int st = oracle_segment_pair_inductance(a0, a1, b0, b1, rw, (k == l && i == j), &m);
          if (st > status) status = st;
          s += m;
        }
      }
      M[k * n_loops + l] = s;
    }
  }
  return status;
}

/* ------------------------------------------------------------------------------------
 * Port system (Eq. 2, Eq. 11): A = diag(R) + j w M + diag(1/(j w C)).
 * ------------------------------------------------------------------------------------ */
void oracle_assemble(int32_t n, const double* M, const double* R, double omega,
                     const double* C, double complex* A) {
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t j = 0; j < n; ++j) A[i * n + j] = I * omega * M[i * n + j];
    A[i * n + i] += R[i] + 1.0 / (I * omega * C[i]);
  }
}

/* Dense LU with partial pivoting, in place: P A = L U with unit lower L below the
 * diagonal and U on and above it. piv[k] = the row swapped with row k at step k.
 * The pivot is the first row of maximal modulus (cabs) in column k at or below row k.
 * Returns 1 if a zero pivot occurs, else 0. */
int oracle_lu(int32_t n, double complex* A, int32_t* piv) {
  for (int32_t k = 0; k < n; ++k) {
    int32_t p = k;
    double best = cabs(A[k * n + k]);
    for (int32_t i = k + 1; i < n; ++i) {
      double v = cabs(A[i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k) {
      for (int32_t j = 0; j < n; ++j) {
        double complex t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    }
    for (int32_t i = k + 1; i < n; ++i) {
      double complex l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int32_t j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return 0;
}

/* Solve A x = b with the factors of oracle_lu; b is overwritten with x. */
void oracle_lu_solve(int32_t n, const double complex* LU, const int32_t* piv,
                     double complex* b) {
  for (int32_t k = 0; k < n; ++k) {
    if (piv[k] != k) {
      double complex t = b[k];
      b[k] = b[piv[k]];
      b[piv[k]] = t;
    }
  }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
  for (int32_t i = n - 1; i >= 0; --i) {
    for (int32_t j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
    b[i] /= LU[i * n + i];
  }
}

/* General impedance-route solve (the Z form of Eq. 4-6): (Z + diag(Zload)) I = V.
 * Z, Zload, V complex; I written to Iout. Returns the LU status. */
int oracle_solve_loaded(int32_t n, const double complex* Z, const double complex* Zload,
                        const double complex* V, double complex* Iout) {
  double complex* A = malloc(sizeof(double complex) * (size_t)n * n);
  int32_t* piv = malloc(sizeof(int32_t) * (size_t)n);
  memcpy(A, Z, sizeof(double complex) * (size_t)n * n);
  for (int32_t i = 0; i < n; ++i) A[i * n + i] += Zload[i];
  int st = oracle_lu(n, A, piv);
  if (st == 0) {
    memcpy(Iout, V, sizeof(double complex) * (size_t)n);
    oracle_lu_solve(n, A, piv, Iout);
  }
  free(A);
  free(piv);
  return st;
}

/* ------------------------------------------------------------------------------------
 * Objective (Eq. 1) and its derivative with respect to the field.
 *   mode 0 (magnitude, as optimised in Sec. IV-C): e = (|b| - t)^2,
 *          G = d e/d Re b + j d e/d Im b = 2 (|b| - t) b/|b| (0 when b = 0);
 *   mode 1 (complex target): e = |b - t|^2, G = 2 (b - t).
 * The loss of one (configuration, structure) is the mean of e over its frequencies and
 * loss points (our reading: Eq. 1 names a mean squared error without fixing how
 * frequencies enter).
 * ------------------------------------------------------------------------------------ */
static double oracle_point_loss(int mode, double complex b, const double* t, double complex* G) {
  if (mode == 0) {
    double a = cabs(b);
    double r = a - t[0];
    *G = (a > 0.0) ? 2.0 * r * b / a : 0.0;
    return r * r;
  }
  double complex tc = t[0] + I * t[1];
  double complex e = b - tc;
  *G = 2.0 * e;
  return creal(e) * creal(e) + cimag(e) * cimag(e);
}

/* Objective term of one loss point with an optional weight w and complex offset o
 * (NULL: 1 and 0), evaluated on w (b + o). This is the signal-enhancement objective of
 * Sec. IV-B: the enhancement at a point is beta = |B_MTS| / |B_ref|, the field with the
 * structure (its induced field b plus the C-independent incident field o) over the field of a
 * reference run without it, so (beta - beta_target)^2 is the magnitude term of w (b + o) with
 * w = 1/|B_ref| and target beta_target. G, the derivative with respect to b, is w times the
 * derivative with respect to w (b + o). */
static double oracle_objective_term(int mode, double complex b, const double* t,
                                    const double* weight, const double complex* offset,
                                    int64_t i, double complex* G) {
  const double w = weight ? weight[i] : 1.0;
  const double complex bb = (offset ? b + offset[i] : b) * w;
  const double e = oracle_point_loss(mode, bb, t, G);
  *G *= w;
  return e;
}

/* ------------------------------------------------------------------------------------
 * Forward map of one structure for a batch of configurations (Eq. 2, 6-7, 11, 1).
 *   N loops, P points, H[P][N], M[N][N], R[N]
 *   n_cfg configurations, C[b][N] (farad)
 *   F frequencies omega[F] (rad/s), drive V[F][N] complex
 *   loss points loss_idx[L] (indices into the P points)
 *   target: mode 0 real [F][L]; mode 1 complex [F][L]; per configuration when
 *           target_per_cfg != 0 ([n_cfg][F][L]).
 * Outputs (each nullable): I_out[b][f][N], B_out[b][f][P], loss_out[b].
 * Configurations are independent; the loop over them may run in parallel threads.
 * Returns the number of singular systems.
 * ------------------------------------------------------------------------------------ */
int oracle_forward_w(int32_t N, int64_t P, const double* H, const double* M, const double* R,
                     int64_t n_cfg, const double* C, int32_t F, const double* omega,
                     const double complex* V, int32_t L, const int64_t* loss_idx,
                     const double* target, int32_t target_per_cfg, int32_t mode,
                     const double* weight, const double complex* offset,
                     double complex* I_out, double complex* B_out, double* loss_out) {
  int n_bad = 0;
  const int64_t tw = (mode == 0) ? 1 : 2;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_cfg; ++b) {
    double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double acc = 0.0;
    for (int32_t f = 0; f < F; ++f) {
      oracle_assemble(N, M, R, omega[f], C + b * N, A);
      if (oracle_lu(N, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      memcpy(x, V + (int64_t)f * N, sizeof(double complex) * (size_t)N);
      oracle_lu_solve(N, A, piv, x);
      if (I_out) memcpy(I_out + (b * F + f) * N, x, sizeof(double complex) * (size_t)N);
      if (B_out) {
        for (int64_t p = 0; p < P; ++p) {
          double complex s = 0.0;
          for (int32_t k = 0; k < N; ++k) s += H[p * N + k] * x[k];
          B_out[(b * F + f) * P + p] = s;
        }
      }
      if (loss_out) {
        const double* t = target + (target_per_cfg ? b * (int64_t)F * L * tw : 0);
        for (int32_t l = 0; l < L; ++l) {
          double complex s = 0.0, G;
          for (int32_t k = 0; k < N; ++k) s += H[loss_idx[l] * N + k] * x[k];
          acc += oracle_objective_term(mode, s, t + ((int64_t)f * L + l) * tw, weight, offset,
                                       (int64_t)f * L + l, &G);
        }
      }
    }
    if (loss_out) loss_out[b] = (F * L > 0) ? acc / ((double)F * L) : 0.0;
    free(A);
    free(piv);
    free(x);
  }
  return n_bad;
}

int oracle_forward(int32_t N, int64_t P, const double* H, const double* M, const double* R,
                   int64_t n_cfg, const double* C, int32_t F, const double* omega,
                   const double complex* V, int32_t L, const int64_t* loss_idx,
                   const double* target, int32_t target_per_cfg, int32_t mode,
                   double complex* I_out, double complex* B_out, double* loss_out) {
  return oracle_forward_w(N, P, H, M, R, n_cfg, C, F, omega, V, L, loss_idx, target,
                          target_per_cfg, mode, NULL, NULL, I_out, B_out, loss_out);
}

/* ------------------------------------------------------------------------------------
 * Gradient of the loss with respect to C, adjoint form.
 * Eq. 9 applied to the impedance route: dI = -A^-1 dA I with dA_kk/dC_k = j/(w C_k^2)
 * (the derivative of 1/(j w C_k)). For a real loss of b = H I with
 * G = dloss/dRe b + j dloss/dIm b, dloss = Re(sum_l conj(G_l) db_l) = Re(u^T dI) with
 * u = H_loss^T conj(G). A is complex symmetric (M symmetric), so with mu = A^-1 u,
 *   dloss/dC_k = -Re(mu_k j I_k/(w C_k^2)) = Im(mu_k I_k)/(w C_k^2),
 * summed over frequencies and divided by the same F*L as the loss.
 * Writes grad_out[b][N]. Returns the number of singular systems.
 * ------------------------------------------------------------------------------------ */
int oracle_gradient_adjoint_w(int32_t N, int64_t P, const double* H, const double* M,
                              const double* R, int64_t n_cfg, const double* C, int32_t F,
                              const double* omega, const double complex* V, int32_t L,
                              const int64_t* loss_idx, const double* target,
                              int32_t target_per_cfg, int32_t mode, const double* weight,
                              const double complex* offset, double* grad_out) {
  (void)P;
  int n_bad = 0;
  const int64_t tw = (mode == 0) ? 1 : 2;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_cfg; ++b) {
    double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* mu = malloc(sizeof(double complex) * (size_t)N);
    const double* Cb = C + b * N;
    for (int32_t k = 0; k < N; ++k) grad_out[b * N + k] = 0.0;
    for (int32_t f = 0; f < F; ++f) {
      oracle_assemble(N, M, R, omega[f], Cb, A);
      if (oracle_lu(N, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      memcpy(x, V + (int64_t)f * N, sizeof(double complex) * (size_t)N);
      oracle_lu_solve(N, A, piv, x);
      const double* t = target + (target_per_cfg ? b * (int64_t)F * L * tw : 0);
      for (int32_t k = 0; k < N; ++k) mu[k] = 0.0;
      for (int32_t l = 0; l < L; ++l) {
        double complex s = 0.0, G;
        for (int32_t k = 0; k < N; ++k) s += H[loss_idx[l] * N + k] * x[k];
        oracle_objective_term(mode, s, t + ((int64_t)f * L + l) * tw, weight, offset,
                              (int64_t)f * L + l, &G);
        for (int32_t k = 0; k < N; ++k) mu[k] += H[loss_idx[l] * N + k] * conj(G);
      }
      oracle_lu_solve(N, A, piv, mu); /* A^T = A */
      for (int32_t k = 0; k < N; ++k)
        grad_out[b * N + k] += cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);
    }
    for (int32_t k = 0; k < N; ++k)
      grad_out[b * N + k] = (F * L > 0) ? grad_out[b * N + k] / ((double)F * L) : 0.0;
    free(A);
    free(piv);
    free(x);
    free(mu);
  }
  return n_bad;
}

int oracle_gradient_adjoint(int32_t N, int64_t P, const double* H, const double* M,
                            const double* R, int64_t n_cfg, const double* C, int32_t F,
                            const double* omega, const double complex* V, int32_t L,
                            const int64_t* loss_idx, const double* target,
                            int32_t target_per_cfg, int32_t mode, double* grad_out) {
  return oracle_gradient_adjoint_w(N, P, H, M, R, n_cfg, C, F, omega, V, L, loss_idx, target,
                                   target_per_cfg, mode, NULL, NULL, grad_out);
}

/* Gradients of the same objective with respect to the loop resistances R_k and the self
 * inductances L_k = M_kk (Fig. 2 names R and L as optimisation variables beside C). From
 * d(A^-1) = -A^-1 dA A^-1 (Eq. 8-9) with dA/dR_k = e_k e_k^T and dA/dM_kk = j w e_k e_k^T:
 *   dloss/dR_k = -Re(mu_k I_k),   dloss/dL_k = -Re(j w mu_k I_k) = w Im(mu_k I_k),
 * summed over frequencies and divided by F*L like the loss. Writes gR[b][N], gL[b][N].
 * Returns the number of singular systems. */
int oracle_gradient_rl(int32_t N, const double* H, const double* M, const double* R,
                       int64_t n_cfg, const double* C, int32_t F, const double* omega,
                       const double complex* V, int32_t L, const int64_t* loss_idx,
                       const double* target, int32_t target_per_cfg, int32_t mode, double* gR,
                       double* gL) {
  int n_bad = 0;
  const int64_t tw = (mode == 0) ? 1 : 2;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_cfg; ++b) {
    double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* mu = malloc(sizeof(double complex) * (size_t)N);
    const double* Cb = C + b * N;
    for (int32_t k = 0; k < N; ++k) gR[b * N + k] = gL[b * N + k] = 0.0;
    for (int32_t f = 0; f < F; ++f) {
      oracle_assemble(N, M, R, omega[f], Cb, A);
      if (oracle_lu(N, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      memcpy(x, V + (int64_t)f * N, sizeof(double complex) * (size_t)N);
      oracle_lu_solve(N, A, piv, x);
      const double* t = target + (target_per_cfg ? b * (int64_t)F * L * tw : 0);
      for (int32_t k = 0; k < N; ++k) mu[k] = 0.0;
      for (int32_t l = 0; l < L; ++l) {
        double complex s = 0.0, G;
        for (int32_t k = 0; k < N; ++k) s += H[loss_idx[l] * N + k] * x[k];
        oracle_point_loss(mode, s, t + ((int64_t)f * L + l) * tw, &G);
        for (int32_t k = 0; k < N; ++k) mu[k] += H[loss_idx[l] * N + k] * conj(G);
      }
      oracle_lu_solve(N, A, piv, mu); /* A^T = A */
      for (int32_t k = 0; k < N; ++k) {
        gR[b * N + k] += -creal(mu[k] * x[k]);
        gL[b * N + k] += omega[f] * cimag(mu[k] * x[k]);
      }
    }
    const double nrm = (F * L > 0) ? 1.0 / ((double)F * L) : 0.0;
    for (int32_t k = 0; k < N; ++k) {
      gR[b * N + k] *= nrm;
      gL[b * N + k] *= nrm;
    }
    free(A);
    free(piv);
    free(x);
    free(mu);
  }
  return n_bad;
}

/* Gradients of the same objective with respect to the angular frequencies w_f (with the
 * drive V held fixed) and to the drive V itself. With mu = A^-1 H_loss^T conj(G) as above:
 *   dA/dw = j M + diag(j / (w^2 C))  (d(1/(j w C))/dw = -1/(j w^2 C)), so
 *   dloss/dw_f = -Re(mu^T dA/dw I) = Im(mu^T M I) + sum_k Im(mu_k I_k) / (w^2 C_k);
 *   dI = A^-1 dV gives dloss = Re(mu^T dV), i.e. the cotangent dL/dRe V + j dL/dIm V =
 *   conj(mu). Both divided by F*L like the loss. Writes gw[b][F] and gV[b][F][N] (complex).
 * Returns the number of singular systems. */
int oracle_gradient_omega_v(int32_t N, const double* H, const double* M, const double* R,
                            int64_t n_cfg, const double* C, int32_t F, const double* omega,
                            const double complex* V, int32_t L, const int64_t* loss_idx,
                            const double* target, int32_t target_per_cfg, int32_t mode,
                            double* gw, double complex* gV) {
  int n_bad = 0;
  const int64_t tw = (mode == 0) ? 1 : 2;
  const double nrm = (F * L > 0) ? 1.0 / ((double)F * L) : 0.0;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_cfg; ++b) {
    double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* mu = malloc(sizeof(double complex) * (size_t)N);
    const double* Cb = C + b * N;
    for (int32_t f = 0; f < F; ++f) {
      gw[b * F + f] = 0.0;
      for (int32_t k = 0; k < N; ++k) gV[(b * F + f) * N + k] = 0.0;
      oracle_assemble(N, M, R, omega[f], Cb, A);
      if (oracle_lu(N, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      memcpy(x, V + (int64_t)f * N, sizeof(double complex) * (size_t)N);
      oracle_lu_solve(N, A, piv, x);
      const double* t = target + (target_per_cfg ? b * (int64_t)F * L * tw : 0);
      for (int32_t k = 0; k < N; ++k) mu[k] = 0.0;
      for (int32_t l = 0; l < L; ++l) {
        double complex s = 0.0, G;
        for (int32_t k = 0; k < N; ++k) s += H[loss_idx[l] * N + k] * x[k];
        oracle_point_loss(mode, s, t + ((int64_t)f * L + l) * tw, &G);
        for (int32_t k = 0; k < N; ++k) mu[k] += H[loss_idx[l] * N + k] * conj(G);
      }
      oracle_lu_solve(N, A, piv, mu); /* A^T = A */
      const double w = omega[f];
      double complex muMI = 0.0;
      double diag = 0.0;
      for (int32_t k = 0; k < N; ++k) {
        double complex MI = 0.0;
        for (int32_t l = 0; l < N; ++l) MI += M[k * N + l] * x[l];
        muMI += mu[k] * MI;
        diag += cimag(mu[k] * x[k]) / (w * w * Cb[k]);
        gV[(b * F + f) * N + k] = conj(mu[k]) * nrm;
      }
      gw[b * F + f] = (cimag(muMI) + diag) * nrm;
    }
    free(A);
    free(piv);
    free(x);
    free(mu);
  }
  return n_bad;
}

/* Gradient with respect to C for an arbitrary field cotangent (the torch convention
 * gB = dL/dRe B + j dL/dIm B over the full field B[b][f][P]):
 * dL/dC_k = sum_f Im(mu_k I_k)/(w C_k^2) with mu = A^-1 H^T conj(gB[b][f]). */
int oracle_gradient_field(int32_t N, int64_t P, const double* H, const double* M,
                          const double* R, int64_t n_cfg, const double* C, int32_t F,
                          const double* omega, const double complex* V,
                          const double complex* gB, double* grad_out) {
  int n_bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_cfg; ++b) {
    double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
    double complex* x = malloc(sizeof(double complex) * (size_t)N);
    double complex* mu = malloc(sizeof(double complex) * (size_t)N);
    const double* Cb = C + b * N;
    for (int32_t k = 0; k < N; ++k) grad_out[b * N + k] = 0.0;
    for (int32_t f = 0; f < F; ++f) {
      oracle_assemble(N, M, R, omega[f], Cb, A);
      if (oracle_lu(N, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      memcpy(x, V + (int64_t)f * N, sizeof(double complex) * (size_t)N);
      oracle_lu_solve(N, A, piv, x);
      for (int32_t k = 0; k < N; ++k) {
        double complex s = 0.0;
        for (int64_t p = 0; p < P; ++p) s += H[p * N + k] * conj(gB[(b * F + f) * P + p]);
        mu[k] = s;
      }
      oracle_lu_solve(N, A, piv, mu);
      for (int32_t k = 0; k < N; ++k)
        grad_out[b * N + k] += cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);
    }
    free(A);
    free(piv);
    free(x);
    free(mu);
  }
  return n_bad;
}

/* Direct-form derivative of the currents (Eq. 8-9 in the impedance route), one extra
 * solve per capacitor: dI/dC_k = -A^-1 e_k (j/(w C_k^2)) I_k. For one configuration
 * and one frequency; dI_out[k][i] = dI_i/dC_k. Returns the LU status. */
int oracle_dcurrents_dC(int32_t N, const double* M, const double* R, double omega,
                        const double* C, const double complex* V, double complex* dI_out) {
  double complex* A = malloc(sizeof(double complex) * (size_t)N * N);
  int32_t* piv = malloc(sizeof(int32_t) * (size_t)N);
  double complex* x = malloc(sizeof(double complex) * (size_t)N);
  oracle_assemble(N, M, R, omega, C, A);
  int st = oracle_lu(N, A, piv);
  if (st == 0) {
    memcpy(x, V, sizeof(double complex) * (size_t)N);
    oracle_lu_solve(N, A, piv, x);
    for (int32_t k = 0; k < N; ++k) {
      double complex* col = dI_out + (int64_t)k * N;
      for (int32_t i = 0; i < N; ++i) col[i] = 0.0;
      col[k] = -(I / (omega * C[k] * C[k])) * x[k];
      oracle_lu_solve(N, A, piv, col);
    }
  }
  free(A);
  free(piv);
  free(x);
  return st;
}

/* ------------------------------------------------------------------------------------
 * Scattering-parameter route (Eq. 3-7), used to cross-check the impedance route.
 * Structure with n ports and impedance matrix Z (complex n x n). Port `drive` connects to
 * an external source with reference impedance Z0 and outgoing wave sqrt(Z0 P) (Eq. 4,
 * S_C11[drive][drive] = 0, S_C12 = e_drive); every other port k is terminated by Zload[k]
 * with reflection (Zload - Z0)/(Zload + Z0) (Eq. 3).
 *   S0 = (Z - Z0 1)(Z + Z0 1)^-1
 *   A  = 1 - S_C11 S0,   V+ = A^-1 S_C12 sqrt(Z0 P)          (Eq. 6)
 *   port currents I = (1 - S0) V+ / Z0                         (waves V+- = (V +- Z0 I)/2)
 * Writes I_out[n]. If dI_out is not NULL it also writes, from Eq. 10 with
 * dS_C12/dC = 0 and dS_C11/dC_k = e_k e_k^T dGamma_k/dZload_k dZload_k/dC_k where the
 * load is a capacitor in series with the rest of Zload (dZload_k/dC_k = j/(w C_k^2),
 * dGamma/dZload = 2 Z0/(Zload + Z0)^2):
 *   dV+/dC_k = A^-1 dS_C11/dC_k S0 V+,  dI/dC_k = (1 - S0) dV+/dC_k / Z0,
 * as dI_out[k][i] for the non-drive ports k (C given per port, C[drive] ignored).
 * Returns the LU status.
 * ------------------------------------------------------------------------------------ */
int oracle_sroute(int32_t n, const double complex* Z, const double complex* Zload,
                  int32_t drive, double Z0, double P_in, double omega, const double* C,
                  double complex* I_out, double complex* dI_out) {
  size_t nn = (size_t)n * n;
  double complex* Zp = malloc(sizeof(double complex) * nn);
  double complex* S0 = malloc(sizeof(double complex) * nn);
  double complex* Am = malloc(sizeof(double complex) * nn);
  double complex* gam = malloc(sizeof(double complex) * (size_t)n);
  double complex* vp = malloc(sizeof(double complex) * (size_t)n);
  double complex* tmp = malloc(sizeof(double complex) * (size_t)n);
  int32_t* piv = malloc(sizeof(int32_t) * (size_t)n);
  int st = 0;
  /* S0 = (Z - Z0)(Z + Z0)^-1: solve S0 (Z + Z0) = (Z - Z0), i.e. (Z + Z0)^T S0^T = (Z - Z0)^T */
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) Zp[i * n + j] = Z[j * n + i] + (i == j ? Z0 : 0.0);
  st = oracle_lu(n, Zp, piv);
  if (st) goto done;
  for (int32_t i = 0; i < n; ++i) {
    /* row i of S0 = column i of S0^T = solve (Z+Z0)^T s = (Z - Z0)^T e_i -> row i of Z - Z0 */
    for (int32_t j = 0; j < n; ++j) tmp[j] = Z[i * n + j] - (i == j ? Z0 : 0.0);
    oracle_lu_solve(n, Zp, piv, tmp);
    for (int32_t j = 0; j < n; ++j) S0[i * n + j] = tmp[j];
  }
  for (int32_t k = 0; k < n; ++k)
    gam[k] = (k == drive) ? 0.0 : (Zload[k] - Z0) / (Zload[k] + Z0); /* Eq. 3 */
  /* A = 1 - S_C11 S0 (S_C11 diagonal) */
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) Am[i * n + j] = (i == j ? 1.0 : 0.0) - gam[i] * S0[i * n + j];
  st = oracle_lu(n, Am, piv);
  if (st) goto done;
  for (int32_t i = 0; i < n; ++i) vp[i] = (i == drive) ? csqrt(Z0 * P_in) : 0.0; /* Eq. 4 */
  oracle_lu_solve(n, Am, piv, vp);                                                /* Eq. 6 */
  for (int32_t i = 0; i < n; ++i) {
    double complex s = vp[i];
    for (int32_t j = 0; j < n; ++j) s -= S0[i * n + j] * vp[j];
    I_out[i] = s / Z0;
  }
  if (dI_out) {
    for (int32_t k = 0; k < n; ++k) {
      double complex* col = dI_out + (int64_t)k * n;
      for (int32_t i = 0; i < n; ++i) col[i] = 0.0;
      if (k == drive) continue;
      double complex zl = Zload[k];
      double complex dgam = 2.0 * Z0 / ((zl + Z0) * (zl + Z0)) * (I / (omega * C[k] * C[k]));
      double complex sv = 0.0; /* (S0 V+)_k */
      for (int32_t j = 0; j < n; ++j) sv += S0[k * n + j] * vp[j];
      for (int32_t i = 0; i < n; ++i) tmp[i] = 0.0;
      tmp[k] = dgam * sv; /* Eq. 10 inner bracket */
      oracle_lu_solve(n, Am, piv, tmp);
      for (int32_t i = 0; i < n; ++i) {
        double complex s = tmp[i];
        for (int32_t j = 0; j < n; ++j) s -= S0[i * n + j] * tmp[j];
        col[i] = s / Z0;
      }
    }
  }
done:
  free(Zp);
  free(S0);
  free(Am);
  free(gam);
  free(vp);
  free(tmp);
  free(piv);
  return st;
}

/* ------------------------------------------------------------------------------------
 * The scattering-parameter pipeline as a first-class path (Sec. III and III-A, Eq. 3-7,
 * Eq. 10), on a structure described by its own S-matrix S0 and per-port fields, both from
 * any solver.
 *
 *   n0 structure ports, n1 external ports, n = n0 + n1; F frequencies; P field points.
 *   S0[f]      complex [n0][n0]   structure scattering matrix (Eq. 5: V-res = S0 V+res)
 *   field[f]   complex [P][n0]    field at point p when port k receives a unit incident
 *                                 wave (Eq. 7's B, one component per point)
 *   Sconst[f]  complex [n][n]     constant part of the network tensor S_C (Sec. III-A 2)
 *   svar[b][f] complex [nS]       user-preprocessed variable S-parameters; entry i goes to
 *                                 row rows[i], column cols[i] of S_C,var (Sec. III-A 1)
 * Per configuration b and frequency f (Sec. III-A 3, Eq. 6, Eq. 7):
 *   S_C = S_C,var + S_C,const;  S11 = S_C[0:n0, 0:n0],  S12 = S_C[0:n0, n0:n]
 *   A = 1 - S11 S0;  W = A^-1 S12  (the wave ratio V+res / V-exc, n0 x n1)
 *   Bcomb[b][c][f][p] = sum_k field[f][p][k] W[k][c]
 * Objective: the point loss of oracle_point_loss on Bcomb at the loss points, target
 * [f][c][l] (mode 0 real, mode 1 complex), mean over (f, c, l); optional weight and offset
 * [f][c][l] as in oracle_objective_term (the enhancement objective of Sec. IV-B).
 * ------------------------------------------------------------------------------------ */
static void oracle_sroute_assemble(int32_t n0, int32_t n1, int32_t nS, const int32_t* rows,
                                   const int32_t* cols, const double complex* S0,
                                   const double complex* Sconst, const double complex* svar,
                                   double complex* SC, double complex* A) {
  const int32_t n = n0 + n1;
  memcpy(SC, Sconst, sizeof(double complex) * (size_t)n * n);
  for (int32_t i = 0; i < nS; ++i) SC[rows[i] * n + cols[i]] += svar[i];
  for (int32_t i = 0; i < n0; ++i)
    for (int32_t j = 0; j < n0; ++j) {
      double complex s = 0.0;
      for (int32_t k = 0; k < n0; ++k) s += SC[i * n + k] * S0[k * n0 + j];
      A[i * n0 + j] = (i == j ? 1.0 : 0.0) - s;
    }
}

/* W = A^-1 S12 column by column with the factors of A; W is [n0][n1]. */
static void oracle_sroute_wave_ratio(int32_t n0, int32_t n1, const double complex* LU,
                                     const int32_t* piv, const double complex* SC,
                                     double complex* col, double complex* W) {
  const int32_t n = n0 + n1;
  for (int32_t c = 0; c < n1; ++c) {
    for (int32_t k = 0; k < n0; ++k) col[k] = SC[k * n + n0 + c];
    oracle_lu_solve(n0, LU, piv, col);
    for (int32_t k = 0; k < n0; ++k) W[k * n1 + c] = col[k];
  }
}

int oracle_sroute_forward(int32_t n0, int32_t n1, int32_t F, int64_t P, int32_t nS,
                          const int32_t* rows, const int32_t* cols, const double complex* S0,
                          const double complex* field, const double complex* Sconst,
                          int64_t n_batch, const double complex* svar, int32_t L,
                          const int64_t* loss_idx, const double* target, int32_t mode,
                          const double* weight, const double complex* offset,
                          double complex* W_out, double complex* B_out, double* loss_out) {
  const int32_t n = n0 + n1;
  const int64_t tw = (mode == 0) ? 1 : 2;
  int n_bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_batch; ++b) {
    double complex* SC = malloc(sizeof(double complex) * (size_t)n * n);
    double complex* A = malloc(sizeof(double complex) * (size_t)n0 * n0);
    double complex* W = malloc(sizeof(double complex) * (size_t)n0 * n1);
    double complex* col = malloc(sizeof(double complex) * (size_t)n0);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)n0);
    double acc = 0.0;
    for (int32_t f = 0; f < F; ++f) {
      oracle_sroute_assemble(n0, n1, nS, rows, cols, S0 + (int64_t)f * n0 * n0,
                             Sconst + (int64_t)f * n * n, svar + (b * F + f) * nS, SC, A);
      if (oracle_lu(n0, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      oracle_sroute_wave_ratio(n0, n1, A, piv, SC, col, W);
      if (W_out) memcpy(W_out + (b * F + f) * n0 * n1, W, sizeof(double complex) * (size_t)n0 * n1);
      const double complex* fd = field + (int64_t)f * P * n0;
      for (int32_t c = 0; c < n1; ++c) {
        if (B_out)
          for (int64_t p = 0; p < P; ++p) {
            double complex s = 0.0;
            for (int32_t k = 0; k < n0; ++k) s += fd[p * n0 + k] * W[k * n1 + c];
            B_out[((b * n1 + c) * F + f) * P + p] = s;
          }
        if (loss_out)
          for (int32_t l = 0; l < L; ++l) {
            double complex s = 0.0, G;
            for (int32_t k = 0; k < n0; ++k) s += fd[loss_idx[l] * n0 + k] * W[k * n1 + c];
            const int64_t i = ((int64_t)f * n1 + c) * L + l;
            acc += oracle_objective_term(mode, s, target + i * tw, weight, offset, i, &G);
          }
      }
    }
    if (loss_out) loss_out[b] = (F * n1 * L > 0) ? acc / ((double)F * n1 * L) : 0.0;
    free(SC);
    free(A);
    free(W);
    free(col);
    free(piv);
  }
  return n_bad;
}

/* Gradient of the objective with respect to the variable S-parameters, from Eq. 10 in
 * forward mode: entry i enters S_C at (r, c) = (rows[i], cols[i]), so d S_C / d svar_i is
 * the unit matrix E_rc (S_C is holomorphic in svar). Eq. 10 gives
 *   dW = A^-1 (dS11 S0 W + dS12):   r < n0, c < n0:  row r of the bracket is row c of S0 W;
 *                                    r < n0, c >= n0: the bracket is E_{r, c-n0};
 *                                    r >= n0:         S21 and S22 do not reach the field.
 * With dBcomb = field dW and G the objective's field derivative (oracle_point_loss), the
 * gradient in torch's convention dL/dRe + j dL/dIm of a holomorphic dependence is
 *   grad_i = sum over (f, c, l) of conj(dBcomb_l,c) G_l,c / (F n1 L).
 * One extra solve per variable and frequency. Writes grad_out[b][f][nS]. */
int oracle_sroute_gradient(int32_t n0, int32_t n1, int32_t F, int64_t P, int32_t nS,
                           const int32_t* rows, const int32_t* cols, const double complex* S0,
                           const double complex* field, const double complex* Sconst,
                           int64_t n_batch, const double complex* svar, int32_t L,
                           const int64_t* loss_idx, const double* target, int32_t mode,
                           const double* weight, const double complex* offset,
                           double complex* grad_out) {
  const int32_t n = n0 + n1;
  const int64_t tw = (mode == 0) ? 1 : 2;
  const double norm = (double)F * n1 * L;
  int n_bad = 0;
  (void)P;
#pragma omp parallel for schedule(static) reduction(+ : n_bad)
  for (int64_t b = 0; b < n_batch; ++b) {
    double complex* SC = malloc(sizeof(double complex) * (size_t)n * n);
    double complex* A = malloc(sizeof(double complex) * (size_t)n0 * n0);
    double complex* W = malloc(sizeof(double complex) * (size_t)n0 * n1);
    double complex* SW = malloc(sizeof(double complex) * (size_t)n0 * n1);
    double complex* G = malloc(sizeof(double complex) * (size_t)(n1 * L > 0 ? n1 * L : 1));
    double complex* col = malloc(sizeof(double complex) * (size_t)n0);
    int32_t* piv = malloc(sizeof(int32_t) * (size_t)n0);
    for (int32_t f = 0; f < F; ++f) {
      double complex* g = grad_out + (b * F + f) * nS;
      for (int32_t i = 0; i < nS; ++i) g[i] = 0.0;
      const double complex* S0f = S0 + (int64_t)f * n0 * n0;
      oracle_sroute_assemble(n0, n1, nS, rows, cols, S0f, Sconst + (int64_t)f * n * n,
                             svar + (b * F + f) * nS, SC, A);
      if (oracle_lu(n0, A, piv) != 0) {
        n_bad += 1;
        continue;
      }
      oracle_sroute_wave_ratio(n0, n1, A, piv, SC, col, W);
      const double complex* fd = field + (int64_t)f * P * n0;
      for (int32_t c = 0; c < n1; ++c)
        for (int32_t l = 0; l < L; ++l) {
          double complex s = 0.0;
          for (int32_t k = 0; k < n0; ++k) s += fd[loss_idx[l] * n0 + k] * W[k * n1 + c];
          const int64_t i = ((int64_t)f * n1 + c) * L + l;
          oracle_objective_term(mode, s, target + i * tw, weight, offset, i, &G[c * L + l]);
        }
      for (int32_t k = 0; k < n0; ++k) /* S0 W */
        for (int32_t c = 0; c < n1; ++c) {
          double complex s = 0.0;
          for (int32_t j = 0; j < n0; ++j) s += S0f[k * n0 + j] * W[j * n1 + c];
          SW[k * n1 + c] = s;
        }
      for (int32_t i = 0; i < nS; ++i) {
        const int32_t r = rows[i], cc = cols[i];
        if (r >= n0) continue;
        for (int32_t c = 0; c < n1; ++c) {
          /* column c of the Eq. 10 bracket, then one solve */
          for (int32_t k = 0; k < n0; ++k) col[k] = 0.0;
          if (cc < n0) col[r] = SW[cc * n1 + c];
          else if (cc - n0 == c) col[r] = 1.0;
          else continue;
          oracle_lu_solve(n0, A, piv, col);
          for (int32_t l = 0; l < L; ++l) {
            double complex db = 0.0;
            for (int32_t k = 0; k < n0; ++k) db += fd[loss_idx[l] * n0 + k] * col[k];
            g[i] += conj(db) * G[c * L + l] / norm;
          }
        }
      }
    }
    free(SC);
    free(A);
    free(W);
    free(SW);
    free(G);
    free(col);
    free(piv);
  }
  return n_bad;
}
