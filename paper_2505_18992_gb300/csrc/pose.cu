// Camera pose update on the device, one thread per view, float64.
//   xi = -lr * g (plain step) or the Adam direction
//   T_cw <- Exp(xi) T_cw, Exp the SE(3) exponential with xi = (rho, phi)
// The gradient is zeroed after use so a captured graph can replay
// render -> backward -> step without host work.
#include "internal.h"
#include "profiler.h"

namespace vpgs {

__device__ void se3_exp(const double xi[6], double R[9], double t[3]) {
    const double *rho = xi, *phi = xi + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double a, b, c;  // R = I + a W + b W^2,  V = I + b W + c W^2
    if (th < 1e-6) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        c = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
        c = (th - sin(th)) / (th2 * th);
    }
    const double W[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double W2[9];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q)
            W2[3 * r + q] = W[3 * r] * W[q] + W[3 * r + 1] * W[3 + q] + W[3 * r + 2] * W[6 + q];
    double Vm[9];
    for (int k = 0; k < 9; ++k) {
        const double I = (k % 4 == 0) ? 1.0 : 0.0;
        R[k] = I + a * W[k] + b * W2[k];
        Vm[k] = I + b * W[k] + c * W2[k];
    }
    for (int r = 0; r < 3; ++r) t[r] = Vm[3 * r] * rho[0] + Vm[3 * r + 1] * rho[1] + Vm[3 * r + 2] * rho[2];
}

__global__ void pose_step_kernel(double *T_cw, double *dpose, double *adam, int V, double lr_rho,
                                 double lr_phi) {
    grid_dep_enter();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double xi[6];
    double *g = dpose + 6 * v;
    if (adam) {
        double *m = adam + 13 * v, *s = m + 6, *step = m + 12;
        const double b1 = 0.9, b2 = 0.999;
        const double k = *step + 1.0;
        *step = k;
        const double c1 = 1.0 - pow(b1, k), c2 = 1.0 - pow(b2, k);
        for (int i = 0; i < 6; ++i) {
            m[i] = b1 * m[i] + (1.0 - b1) * g[i];
            s[i] = b2 * s[i] + (1.0 - b2) * g[i] * g[i];
            const double lr = i < 3 ? lr_rho : lr_phi;
            xi[i] = -lr * (m[i] / c1) / (sqrt(s[i] / c2) + 1e-15);
        }
    } else {
        for (int i = 0; i < 6; ++i) xi[i] = -(i < 3 ? lr_rho : lr_phi) * g[i];
    }
    double R[9], t[3];
    se3_exp(xi, R, t);
    double *T = T_cw + 16 * v;
    double N[12];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 4; ++q) {
            double acc = R[3 * r] * T[q] + R[3 * r + 1] * T[4 + q] + R[3 * r + 2] * T[8 + q];
            if (q == 3) acc += t[r];
            N[4 * r + q] = acc;
        }
    }
    for (int k = 0; k < 12; ++k) T[k] = N[k];
    for (int i = 0; i < 6; ++i) g[i] = 0.0;
}

cudaError_t launch_pose_step(double *T_cw, double *dpose, double *adam, int V, double lr_rho,
                             double lr_phi, cudaStream_t s) {
    VPGS_LAUNCH("pose_step", s, launch_k(pose_step_kernel, (V + 63) / 64, 64, 0, s, T_cw, dpose, adam, V,
                                                                              lr_rho, lr_phi));
    return cudaGetLastError();
}

}  // namespace vpgs
