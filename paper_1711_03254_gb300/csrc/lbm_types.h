// Plain structs shared by the host runtime and the kernels.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace lbm {

// storage type of the per-cell reference density of the shifted formats
using Ref = __half;

// Per-instance parameters in the arithmetic type T (double or float).
template <class T> struct InstParam {
    T nu[2];     // kinematic viscosities (tau_k - 1/2) T0
    T G;         // coupling of Eq. 7
    T rs[2];     // wall potentials rho^s_1, rho^s_2
    T g[3];      // body acceleration
    T rho_in[2]; // INLET densities
    T u_in[3];   // INLET velocity
    T slip;      // fraction of the wall's particles reflected specularly
};

struct Grid {
    int nx, ny, nz;
    int nxy;
    long long n;  // cells per instance
};

}  // namespace lbm
