// Camera pose update on the device, one warp per view, float64.
//   xi = -lr * g (plain step) or the Adam direction
//   T_cw <- Exp(xi) T_cw, Exp the SE(3) exponential with xi = (rho, phi)
// The gradient is zeroed after use so a captured graph can replay
// render -> backward -> step without host work.
#include "internal.h"
#include "profiler.h"

namespace vpgs {

// b1^n and b2^n for a step count n >= 0 by binary exponentiation (at most 2 log2 n
// multiplications per base, both chains interleaved); FP64 on this part is slow,
// and a general pow would cost several times more
__device__ void int_powers(double b1, double b2, double k, double &p1, double &p2) {
    long long n = (long long)k;
    p1 = 1.0;
    p2 = 1.0;
    while (n > 0) {
        if (n & 1) {
            p1 *= b1;
            p2 *= b2;
        }
        b1 *= b1;
        b2 *= b2;
        n >>= 1;
    }
}

// One warp per view: lanes 0-5 take one component of the step xi each, every
// lane then forms the coefficients of Exp(xi), and lanes 0-11 one entry of the
// new [R t] rows each, so the FP64 chain is one component and one entry long.
//   Exp(xi) = [[R, V rho], [0, 1]],  R = I + a W + b W^2,  V = I + b W + c W^2,
//   W = phi^, th = |phi|, a = sin th / th, b = (1 - cos th) / th^2,
//   c = (th - sin th) / th^3 (Taylor terms below th = 1e-6)
__global__ void pose_step_kernel(double *T_cw, double *dpose, double *adam, int V, double lr_rho,
                                 double lr_phi) {
    grid_dep_enter();
    const int v = blockIdx.x;
    const int lane = threadIdx.x;
    if (v >= V) return;
    double *g = dpose + 6 * v;
    double xi_l = 0.0;  // component `lane` of xi (lanes 0-5)
    if (adam) {
        double *m = adam + 13 * v, *sq = m + 6, *step = m + 12;
        const double b1 = 0.9, b2 = 0.999;
        const double k = *step + 1.0;  // a whole number
        double p1, p2;
        int_powers(b1, b2, k, p1, p2);
        const double c1 = 1.0 - p1, c2 = 1.0 - p2;
        if (lane < 6) {
            const double gi = g[lane];
            const double mi = b1 * m[lane] + (1.0 - b1) * gi;
            const double si = b2 * sq[lane] + (1.0 - b2) * gi * gi;
            m[lane] = mi;
            sq[lane] = si;
            const double lr = lane < 3 ? lr_rho : lr_phi;
            xi_l = -lr * (mi / c1) / (sqrt(si / c2) + 1e-15);
        }
        __syncwarp();  // every lane has read the step count
        if (lane == 0) *step = k;
    } else if (lane < 6) {
        xi_l = -(lane < 3 ? lr_rho : lr_phi) * g[lane];
    }
    double xi[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) xi[i] = __shfl_sync(0xffffffffu, xi_l, i);
    const double *rho = xi, *phi = xi + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double a, b, c;
    if (th < 1e-6) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        double sn, cs;
        sincos(th, &sn, &cs);
        a = sn / th;
        b = (1.0 - cs) / th2;
        c = (th - sn) / (th2 * th);
    }
    const double W[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double *T = T_cw + 16 * v;
    // entry (r, q) of the new top rows: R_r . T_col(q) (+ t_r for q = 3)
    const int r = lane >> 2, q = lane & 3;
    double out = 0.0;
    if (lane < 12) {
        double Rr[3], Vr[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double w2 = W[3 * r] * W[j] + W[3 * r + 1] * W[3 + j] + W[3 * r + 2] * W[6 + j];
            const double I = (r == j) ? 1.0 : 0.0;
            Rr[j] = I + a * W[3 * r + j] + b * w2;
            Vr[j] = I + b * W[3 * r + j] + c * w2;
        }
        out = Rr[0] * T[q] + Rr[1] * T[4 + q] + Rr[2] * T[8 + q];
        if (q == 3) out += Vr[0] * rho[0] + Vr[1] * rho[1] + Vr[2] * rho[2];
    }
    __syncwarp();  // every lane has read T and the gradient
    if (lane < 12) T[lane] = out;
    if (lane < 6) g[lane] = 0.0;
}

cudaError_t launch_pose_step(double *T_cw, double *dpose, double *adam, int V, double lr_rho,
                             double lr_phi, cudaStream_t s) {
    VPGS_LAUNCH("pose_step", s, launch_k(pose_step_kernel, V, 32, 0, s, T_cw, dpose, adam, V, lr_rho, lr_phi));
    return cudaGetLastError();
}

}  // namespace vpgs
