// Symmetric tridiagonal eigenproblem in FP64 for one thread (the Ritz step, a5,
// and the Cullum-Willoughby diagnostic), shared by lanczos.cu and diag.cu.
#pragma once

#include "ftlm_internal.cuh"

namespace ftlm {

// Implicit symmetric tridiagonal QR with Wilkinson shift (Golub & Van Loan,
// "Matrix Computations", Sec. 8.3), deflating from the bottom.  Only the first
// row z of the accumulated rotation matrix is kept: the eigenvector matrix of T is
// the product of the rotations, so its first row gives s_{k,1}.
//
// GB300 has a narrow FP64 pipe, so FP64 square roots and divisions are long
// dependent sequences; each rotation uses one reciprocal square root and no
// division, and one thread runs one chain with many chains per CTA, so the
// latency of many chains overlaps.  The arrays of the chains of a CTA are
// interleaved in shared memory: element k of thread i at [k * T + i].
struct Strided {
    double *p;
    int stride;
    __device__ __forceinline__ double &operator[](int k) const { return p[k * stride]; }
};

// [c s; -s c]^T [a; b] = [r; 0] with r = sqrt(a^2 + b^2) >= 0.
__device__ __forceinline__ void givens(double a, double b, double &c, double &s)
{
    const double r2 = fma(a, a, b * b);
    if (r2 == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    const double ir = rsqrt(r2);
    c = a * ir;
    s = -b * ir;
}

__device__ __forceinline__ bool negligible(double e, double d0, double d1)
{
    return fabs(e) <= 0x1p-52 * (fabs(d0) + fabs(d1)) || fabs(e) < 1e-150;
}

// Returns false when the bottom-up deflation has not reached the top after
// max_sweeps QR sweeps (0: 64 n, far more than the few sweeps per eigenvalue that
// the Wilkinson shift needs); d and z then hold no eigendecomposition.
static __device__ bool tridiag_qr(Strided d, Strided e, Strided z, int n, int max_sweeps = 0)
{
    int hi = n - 1;
    if (max_sweeps <= 0) max_sweeps = 64 * n;
    for (int sweep = 0; hi > 0 && sweep < max_sweeps;) {
        if (negligible(e[hi - 1], d[hi - 1], d[hi])) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !negligible(e[lo - 1], d[lo - 1], d[lo])) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        ++sweep;
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double bb = e[hi - 1];
        const double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * sqrt(fma(dd, dd, bb * bb));
        const double mu = d[hi] - bb * (bb / den);
        double x = d[lo] - mu, zz = e[lo];
        for (int k = lo; k < hi; ++k) {
            double c, s;
            givens(x, zz, c, s);
            if (k > lo) e[k - 1] = c * x - s * zz;
            const double a = d[k], b = e[k], cc = d[k + 1];
            const double c2 = c * c, s2 = s * s, cs = c * s;
            d[k] = c2 * a - 2.0 * cs * b + s2 * cc;
            d[k + 1] = s2 * a + 2.0 * cs * b + c2 * cc;
            e[k] = cs * (a - cc) + (c2 - s2) * b;
            if (k < hi - 1) {
                const double en = e[k + 1];
                x = e[k];
                zz = -s * en;
                e[k + 1] = c * en;
            }
            const double z0 = z[k], z1 = z[k + 1];
            z[k] = c * z0 - s * z1;
            z[k + 1] = s * z0 + c * z1;
        }
    }
    // converged when every remaining off-diagonal entry is negligible (the last
    // permitted sweep may have finished the job)
    for (int k = hi - 1; k >= 0; --k) {
        if (!negligible(e[k], d[k], d[k + 1])) return false;
        e[k] = 0.0;
    }
    return true;
}

// Ascending order of d (and z with it), insertion sort (n <= FTLM_MAX_LANCZOS).
__device__ __forceinline__ void sort_ascending(Strided d, Strided z, int n)
{
    for (int k = 1; k < n; ++k) {
        const double dk = d[k], zk = z[k];
        int j = k - 1;
        while (j >= 0 && d[j] > dk) {
            d[j + 1] = d[j];
            z[j + 1] = z[j];
            --j;
        }
        d[j + 1] = dk;
        z[j + 1] = zk;
    }
}

}  // namespace ftlm
