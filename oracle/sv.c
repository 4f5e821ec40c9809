/*
 * O1 in plain C: in-place gate application to a complex128 state vector.
 *
 * TEST INFRASTRUCTURE ONLY (part of the CPU oracle; never linked by the
 * library).  The same definitions as oracle/statevector.py, written for
 * states too large for NumPy's out-of-place tensordot (a 30-qubit state is
 * 16 GiB; this works on it in place, with no second copy):
 *
 *   qubit q = bit q of a basis index;
 *   one-qubit gate U (2x2, row = output): for each index pair (i0, i1) that
 *     differs only in bit q (i0 with the bit 0),
 *       psi'[i_a] = sum_b U[a][b] psi[i_b];
 *   two-qubit gate U (4x4, basis |q0 q1>, q0 the high bit): for each index
 *     quadruple differing only in bits q0, q1, with j = 2 b(q0) + b(q1),
 *       psi'[i_j] = sum_k U[j][k] psi[i_k];
 *   projector |v><v| on qubit q: psi[i] = 0 wherever bit q of i is not v
 *     (a cut edge fixed to v: the edge-breaking insertion of the Method
 *     section).
 *
 * Every output amplitude is computed from its own group of inputs exactly as
 * written above; groups are independent, so they are visited in parallel.
 */
#include <complex.h>
#include <stdint.h>

typedef double _Complex cplx;

/* index with a zero bit inserted at position p */
static inline uint64_t insert0(uint64_t x, int p) {
  return ((x >> p) << (p + 1)) | (x & ((1ULL << p) - 1));
}

void sv_apply_1q(cplx* psi, int n, int q, const double* re, const double* im) {
  const cplx u00 = re[0] + I * im[0], u01 = re[1] + I * im[1];
  const cplx u10 = re[2] + I * im[2], u11 = re[3] + I * im[3];
  const int64_t pairs = (int64_t)1 << (n - 1);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < pairs; ++t) {
    const uint64_t i0 = insert0((uint64_t)t, q), i1 = i0 | (1ULL << q);
    const cplx a0 = psi[i0], a1 = psi[i1];
    psi[i0] = u00 * a0 + u01 * a1;
    psi[i1] = u10 * a0 + u11 * a1;
  }
}

void sv_apply_2q(cplx* psi, int n, int q0, int q1, const double* re, const double* im) {
  cplx U[4][4];
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 4; ++k) U[j][k] = re[4 * j + k] + I * im[4 * j + k];
  const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
  const int64_t quads = (int64_t)1 << (n - 2);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < quads; ++t) {
    const uint64_t base = insert0(insert0((uint64_t)t, lo), hi);
    uint64_t idx[4];
    cplx a[4];
    for (int j = 0; j < 4; ++j) {
      idx[j] = base | ((uint64_t)(j >> 1) << q0) | ((uint64_t)(j & 1) << q1);
      a[j] = psi[idx[j]];
    }
    for (int j = 0; j < 4; ++j) {
      cplx s = 0;
      for (int k = 0; k < 4; ++k) s += U[j][k] * a[k];
      psi[idx[j]] = s;
    }
  }
}

void sv_project(cplx* psi, int n, int q, int v) {
  const int64_t pairs = (int64_t)1 << (n - 1);
  const uint64_t off = v ? 0ULL : (1ULL << q);   /* the member whose bit q is not v */
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < pairs; ++t) psi[insert0((uint64_t)t, q) | off] = 0;
}

/* <a|b> and <b|b> (double sums per thread, then combined) */
void sv_overlap(const cplx* a, const cplx* b, int n, double* out_re, double* out_im, double* out_bb) {
  const int64_t N = (int64_t)1 << n;
  double sr = 0.0, si = 0.0, sb = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sr, si, sb)
  for (int64_t i = 0; i < N; ++i) {
    const cplx p = conj(a[i]) * b[i];
    sr += creal(p);
    si += cimag(p);
    sb += creal(b[i]) * creal(b[i]) + cimag(b[i]) * cimag(b[i]);
  }
  *out_re = sr;
  *out_im = si;
  *out_bb = sb;
}
