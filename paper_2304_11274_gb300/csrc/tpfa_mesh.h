// tpfa_mesh.h -- fields of a general mesh passed from the host to the mesh
// assembly kernel (tpfa_mesh.cu).
#pragma once

namespace tpfa {

// A mesh given as a connection list.  The pattern's row K holds K and every
// cell connected to it, columns ascending; Tc[e] is the transmissibility of
// the connection of entry e (0 on the diagonal).  phi0 holds
// (V_K / dt) phi0_K (the cell volume folded in; read only when c_r != 0).
template <typename Real>
struct MeshFields {
    const long long* row_ptr;
    const int* col;
    const Real* Tc;
    const Real* p;
    const Real* pn;
    const double* mn;  // (V/dt) phi(p^n) rho(p^n)
    const Real* z;
    const Real* phi0;
};

}  // namespace tpfa
