// tpfa_grid.h -- plain structs passed from the host to the TPFA kernels.
#pragma once

#include <stdint.h>

namespace tpfa {

// Structured grid: cell (i, j, k) is element i + nx (j + ny k) of every field.
struct GridGeom {
    int nx, ny, nz;
    int diag;  // 1 with 10-point connectivity (in-plane diagonals), else 0
};

// Fields read by the assembly kernels.  `Real` is float (mixed path) or
// double (FP64 path).  Owned transmissibilities: cell (i, j, k) stores the
// links to (i+1, j, k) in Tx, (i, j+1, k) in Ty, (i, j, k+1) in Tz,
// (i+1, j+1, k) in Tpp and (i-1, j+1, k) in Tmp; a link that leaves the grid
// stores 0 and is never used.
template <typename Real>
struct AsmFields {
    const Real* p;     // iterate p^{n+1}
    const Real* pn;    // previous time step p^n
    const double* mn;  // (V/dt) phi(p^n) rho(p^n)
    const Real* z;     // cell-centre depth
    const Real* phi0;  // reference porosity (read only when c_r != 0)
    const Real* Tx;
    const Real* Ty;
    const Real* Tz;
    const Real* Tpp;
    const Real* Tmp;
};

// Outputs.  vals has the CSR order of the pattern (columns ascending).
template <typename Real>
struct AsmOut {
    double* R;       // N residuals, or nullptr
    Real* vals;      // nnz Jacobian values, or nullptr (residual only)
    double* diag64;  // N FP64 diagonals (mixed path), or nullptr
    unsigned int* status;  // device error word (bit 0: non-finite value)
};

constexpr unsigned int STATUS_NONFINITE = 1u;
constexpr unsigned int STATUS_DEVICE_CHECK = 2u;  // a checked device access was out of range
constexpr unsigned int STATUS_TIMEOUT = 4u;       // a bounded device-side wait ran out

}  // namespace tpfa
