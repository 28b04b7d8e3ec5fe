// Mapped-geometry setup entry points (called by fdst_setup).
#pragma once
#include "../../include/fdst.h"

struct fdst_ctx;

namespace fdst {
// Geometry, separable fit / weighted pencils, CSR assembly, D_V and D_Q (before the FD chains).
fdst_status build_mapped_pre(fdst_ctx *h);
// Attaches the P_D^G scalings to the FD chains (after they are built).
fdst_status build_mapped_post(fdst_ctx *h);
// P_D^G on the identity map with the one-coordinate viscosity family: weighted
// pencils (separable fit), D_V and D_Q; after build_matvec, before the FD chains.
fdst_status build_identity_geo(fdst_ctx *h);
// The one-coordinate family nu(eta_1) = 1 + (k - 1)(1 - cos(2 pi eta_1)) / 2.
double contrast_viscosity(double eta1, double k);
}  // namespace fdst
