// Internal declarations shared by the host numerics and the CUDA translation
// unit of libqp.  Not part of the public ABI (see include/qp.h).
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

#include "../../include/qp.h"

namespace qp {

using cplx = std::complex<double>;

// U = exp(-i H dt) of a Hermitian M x M matrix (row-major), by scaling and
// squaring of the Taylor series.  The short-time system propagator of Eq.
// SysP (hbar = 1).
std::vector<cplx> short_time_propagator(int M, const std::vector<cplx> &H, double dt);
// the same into U[M*M] for M <= 8, without allocating
void short_time_propagator(int M, const cplx *H, double dt, cplx *U);

// Spectral density J(w) of the bath (ohmic part + Eq. sharpSD resonance).
double spectral_density(const qp_bath &b, double w);

// eta_0 .. eta_{n-1}, box double integrals of the bath correlation function.
int eta_from_bath(const qp_bath &b, double dt, int n, std::vector<cplx> &eta);

// Q(j h), j = 0 .. n-1: the double integral of the bath correlation from 0.
int Q_from_bath(const qp_bath &b, double h, int n, std::vector<cplx> &Q);

}  // namespace qp
