// Host-side plan of a solve: geometry, tree structure, workspace layout and task lists.
#pragma once
#include <string>
#include <vector>
#include "kernels.h"

// Bump allocator over the caller's workspace.  In measuring mode it only adds up sizes, so
// the workspace query and the solve share one layout routine.
struct Arena {
    char* base = nullptr;
    size_t off = 0, cap = 0;
    bool measure = true;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = measure ? nullptr : reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// Normalisation and grid of the fast summation.
struct GridChoice {
    int n = 64, M = 16;
    double s = 1.0;        // x' = (x - c) / s
    double c[3] = {0, 0, 0};
    double err_exp = 0.0;  // min(boundary, spectral) exponent achieved
};

// Choose the scale s and the grid length n (M = n / 4) for point sets of radius R (about c)
// and the per-edge widths eta_e: the kernel must be negligible at |x| = tau - eps_B
// (exponent A s^2 with A = (tau - eps_B)^2 / eta_max) and the Fourier tail beyond M must be
// negligible (exponent B / s^2 with B = pi^2 eta_min M^2); s >= 2R / (tau - eps_B) keeps every
// pairwise difference inside the unregularised region (tau = 1/2 on the unit torus).
GridChoice choose_grid(int d, double R, double eta_min, double eta_max, int n_grid_opt, double epsB);
int max_grid(int d);

// Coefficients c_0..c_{2p} of the boundary polynomial kappa_B(a + t) of Eq. (Ker-reg),
// a = tau - eps_B, from the 2p+1 Hermite conditions (values and derivatives 1..p of kappa at
// a, derivatives 1..p zero at tau).  Returns false if the system is singular.
bool boundary_poly(double eta, double tau, double epsB, int p, double* c);

void set_cuda_error(cudaError_t e, const char* what);
void fill_defaults(mot_options& o, const mot_options* in);
