// Mapped-geometry setup entry points (called by fdst_setup).
#pragma once
#include "../../include/fdst.h"

struct fdst_ctx;

namespace fdst {
// Geometry, separable fit / weighted pencils, CSR assembly, D_V and D_Q (before the FD chains).
fdst_status build_mapped_pre(fdst_ctx *h);
// Attaches the P_D^G scalings to the FD chains (after they are built).
fdst_status build_mapped_post(fdst_ctx *h);
}  // namespace fdst
