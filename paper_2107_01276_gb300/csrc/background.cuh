// Argument blocks and launchers of the background-construction kernels
// (background.cu, section 3.3) and of the fluid vorticity they use for
// solution adaptivity.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Vorticity omega_i = sum_{j != i} V_j ((v_j - v_i) dW/dx - (u_j - u_i)
// dW/dy), grad W = grad_i W(r_ij, h_i), V_j = m_j / rho_j, over the fluid
// neighbour lists; |omega| max into *wmax (bits of a non-negative double).
struct VortArgs {
    int n;
    Domain d;
    const double *x, *y, *u, *v, *m, *rho, *h;
    const uint32_t *off, *list;
    double *omega;
    unsigned long long *wmax;
};

// Step 1: boundary and vorticity marking of background particles.
struct BgMarkArgs {
    int n;                          // background particles (construction order)
    Domain d;
    const double *x, *y, *h;
    double *ds;                     // marked particles take ds_min
    uint32_t *mark;                 // 0, 1 (solid in range), 2 (vorticity)
    double ds_min;
    int nw;                         // solid (dummy wall) particles
    Grid wg;
    const double *wx, *wy, *wh;
    int nr;                         // refinement-region markers
    Grid rg;
    const double *rx, *ry, *rh;
    int nf;                         // fluid particles (0: no vorticity marking)
    Grid fg;
    const double *fx, *fy, *fh, *omega;
    const unsigned long long *wmax;
    double vort_k;
    uint32_t *counts;               // [0] marked, [1] of them by vorticity
};

// Step 2: size rule (Jacobi) and the thresholds m_min, m_max of the split.
struct BgSizeArgs {
    int n;
    const uint32_t *off, *list, *mark;
    const double *ds;
    double *ds_out, *mmin, *mmax;
    double Cr, cr3, ds_min, ds_max, rho0;
};

// Eq. h-smoothing (Jacobi).
struct BgSmoothArgs {
    int n;
    const uint32_t *off, *list;
    const double *h;
    double *h_out;
    double Nr;
};

void launch_vorticity(cudaStream_t s, const VortArgs &a);
void launch_bg_mark(cudaStream_t s, const BgMarkArgs &a);
void launch_bg_size(cudaStream_t s, const BgSizeArgs &a);
void launch_bg_hsmooth(cudaStream_t s, const BgSmoothArgs &a);
// min and max of n positive doubles into out[0], out[1] (bits)
void launch_minmax_pos(cudaStream_t s, int n, const double *v,
                       unsigned long long *out);

}  // namespace sph
