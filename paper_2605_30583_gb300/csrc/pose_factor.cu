// Pose factors: generic node-to-node factors beside the reprojection factors (Sec. IV
// of arXiv 2605.30583, factors between nodes such as odometry / pose-graph
// constraints), here the relative pose of two cameras against a measurement:
//   R_ba = R_b R_a^T,  t_ba = t_b - R_ba t_a,
//   r = s * [ Log(R_m^T R_ba) ; t_ba - t_m ].
// The factor count is small next to the observations, so each factor is one thread in
// FP64 (rotations as unit quaternions).  The Jacobian is taken over left tangent
// perturbations R <- Exp(phi) R of both rotations and the two translations:
//   d r_rot / d phi_a = -J_l^-1(r_rot) E,  d r_rot / d phi_b = J_l^-1(r_rot) R_m^T,
//   d r_t / d phi_a = -R_ba [t_a]x,  d r_t / d t_a = -R_ba,
//   d r_t / d phi_b = [R_ba t_a]x,   d r_t / d t_b = I,
// with E = R_m^T R_ba and J_l^-1 the inverse left Jacobian of SO(3), because
// Log(Exp(d) E) = Log(E) + J_l^-1(Log E) d + O(|d|^2).  It is stored in these
// coordinates (the camera direction records carry phi = J_l(w) d_w) and mapped to the
// rotation-vector coordinates of g and the preconditioner blocks through J_l.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"
#include "mixed_common.cuh"

namespace gbba {

namespace {

__device__ __forceinline__ void qmul(const double* a, const double* b, double* o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Row-major rotation matrix of a unit quaternion (q0; q1 q2 q3).
__device__ __forceinline__ void quat_matrix(const double* q, double* R) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Rotation vector of a unit quaternion, taken with q0 >= 0: 2 atan2(|q_v|, q0) q_v / |q_v|
// (series 2 / q0 (1 - |q_v|^2 / (3 q0^2)) when |q_v| < 1e-7).
__device__ __forceinline__ void quat_log(const double* q, double* w) {
    const double sg = q[0] < 0.0 ? -1.0 : 1.0;
    const double q0 = sg * q[0], q1 = sg * q[1], q2 = sg * q[2], q3 = sg * q[3];
    const double n = sqrt(q1 * q1 + q2 * q2 + q3 * q3);
    const double scale = n > 1e-7 ? 2.0 * atan2(n, q0) / n : (2.0 / q0) * (1.0 - n * n / (3.0 * q0 * q0));
    w[0] = scale * q1;
    w[1] = scale * q2;
    w[2] = scale * q3;
}

// Residual (6) and, if J is not null, the Jacobian J[6][12] over (phi_a, t_a, phi_b,
// t_b) of one factor; rows scaled by the square-root information s.
__device__ void pose_factor(const double* wa, const double* ta, const double* wb, const double* tb,
                            const double* meas, const double* s, double* r, double (*J)[12]) {
    double qa[4], qb[4], qm[4];
    rotvec_quat(wa, qa);
    rotvec_quat(wb, qb);
    rotvec_quat(meas, qm);
    const double qa_c[4] = {qa[0], -qa[1], -qa[2], -qa[3]};
    const double qm_c[4] = {qm[0], -qm[1], -qm[2], -qm[3]};
    double qba[4], qe[4];
    qmul(qb, qa_c, qba);   // R_ba = R_b R_a^T
    qmul(qm_c, qba, qe);   // E = R_m^T R_ba
    double rr[3];
    quat_log(qe, rr);
    double Rba[9];
    quat_matrix(qba, Rba);
    double Rt[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Rt[i] = Rba[3 * i] * ta[0] + Rba[3 * i + 1] * ta[1] + Rba[3 * i + 2] * ta[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r[i] = s[i] * rr[i];
        r[3 + i] = s[3 + i] * (tb[i] - Rt[i] - meas[3 + i]);
    }
    if (J == nullptr) return;
    // J_l^-1(v) = I - [v]x / 2 + c [v]x^2, c = 1/th^2 - (1 + cos th) / (2 th sin th),
    // series 1/12 + th^2/720 + th^4/30240 for th^2 < 1e-6; [v]x^2 = v v^T - th^2 I
    const double th2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
    double c;
    if (th2 < 1e-6) {
        c = 1.0 / 12.0 + th2 * (1.0 / 720.0 + th2 / 30240.0);
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        c = 1.0 / th2 - (1.0 + cs) / (2.0 * th * sn);
    }
    const double K[9] = {0.0, -rr[2], rr[1], rr[2], 0.0, -rr[0], -rr[1], rr[0], 0.0};
    double Ji[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Ji[3 * i + j] = (i == j ? 1.0 - c * th2 : 0.0) - 0.5 * K[3 * i + j] + c * rr[i] * rr[j];
    double E[9], RmT[9];
    quat_matrix(qe, E);
    quat_matrix(qm_c, RmT);
    // [t_a]x and [R_ba t_a]x
    const double Ta[9] = {0.0, -ta[2], ta[1], ta[2], 0.0, -ta[0], -ta[1], ta[0], 0.0};
    const double Tr[9] = {0.0, -Rt[2], Rt[1], Rt[2], 0.0, -Rt[0], -Rt[1], Rt[0], 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double je = 0.0, jm = 0.0, rt = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                je += Ji[3 * i + m] * E[3 * m + j];
                jm += Ji[3 * i + m] * RmT[3 * m + j];
                rt += Rba[3 * i + m] * Ta[3 * m + j];
            }
            J[i][j] = -s[i] * je;
            J[i][3 + j] = 0.0;
            J[i][6 + j] = s[i] * jm;
            J[i][9 + j] = 0.0;
            J[3 + i][j] = -s[3 + i] * rt;
            J[3 + i][3 + j] = -s[3 + i] * Rba[3 * i + j];
            J[3 + i][6 + j] = s[3 + i] * Tr[3 * i + j];
            J[3 + i][9 + j] = i == j ? s[3 + i] : 0.0;
        }
}

__device__ __forceinline__ void load_pose(const float* x, uint32_t c, double* p) {
#pragma unroll
    for (int i = 0; i < 6; ++i) p[i] = (double)x[9 * (size_t)c + i];
}

}  // namespace

// Linearisation of every pose factor at the current parameters, before k_linearize
// (same modes; it reads the camera records of the same point): stores J_f, adds
// J_f^T r to g and the pose part of J_f^T J_f to the camera blocks (rotation columns
// mapped through the record's J_l), and writes 1/2 sum |r_f|^2 to st->fac_cost, which
// k_linearize adds to F.  Mode 2 (evaluation) does the same, as the observations do:
// the normal operator of ba_apply_normal works on that linearisation.
__global__ void k_factor_linearize(Views<float> v, int mode) {
    DevState* st = v.st;
    if (mode == 1 && st->relin == 0) return;
    double cost = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < v.n_fac; k += gridDim.x * blockDim.x) {
        const uint32_t cam[2] = {v.fac_cam[2 * (size_t)k], v.fac_cam[2 * (size_t)k + 1]};
        double pa[6], pb[6], r[6], J[6][12];
        load_pose(v.x, cam[0], pa);
        load_pose(v.x, cam[1], pb);
        pose_factor(pa, pa + 3, pb, pb + 3, v.fac_meas + 6 * (size_t)k, v.fac_sqrt + 6 * (size_t)k, r, J);
#pragma unroll
        for (int i = 0; i < 6; ++i) cost += r[i] * r[i];
        float* Jo = v.fac_J + 72 * (size_t)k;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 12; ++j) Jo[12 * i + j] = (float)J[i][j];
        for (int e = 0; e < 2; ++e) {
            const uint32_t c = cam[e];
            const float* JLf = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
            double Jw[6][6];   // rows of J over this camera's (w, t)
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    Jw[i][j] = J[i][6 * e] * (double)JLf[j] + J[i][6 * e + 1] * (double)JLf[3 + j] +
                               J[i][6 * e + 2] * (double)JLf[6 + j];
                    Jw[i][3 + j] = J[i][6 * e + 3 + j];
                }
            double* g = v.cam_lin + (size_t)c * CL_STRIDE + CL_G;
            float* H = v.cam_H + (size_t)c * CH_STRIDE;
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                double gj = 0.0;
#pragma unroll
                for (int i = 0; i < 6; ++i) gj += Jw[i][j] * r[i];
                atomicAdd(g + j, gj);
#pragma unroll
                for (int l = j; l < 6; ++l) {
                    double hjl = 0.0;
#pragma unroll
                    for (int i = 0; i < 6; ++i) hjl += Jw[i][j] * Jw[i][l];
                    atomicAdd(H + tri_index(9, j, l), (float)hjl);
                }
            }
        }
    }
    double in[1] = {cost}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_FAC], out) && threadIdx.x == 0) st->fac_cost = 0.5 * out[0];
}

// Before k_eval_candidate: 1/2 sum |r_f|^2 at the candidate parameters and |J_f h|^2
// (h's camera direction records from k_candidate), into st->fac_cost_new / fac_jh2.
__global__ void k_factor_eval(Views<float> v) {
    DevState* st = v.st;
    double fnew = 0.0, jh2 = 0.0;
    if (st->lm_active) {
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < v.n_fac; k += gridDim.x * blockDim.x) {
            const uint32_t ca = v.fac_cam[2 * (size_t)k], cb = v.fac_cam[2 * (size_t)k + 1];
            double pa[6], pb[6], r[6];
            load_pose(v.x_new, ca, pa);
            load_pose(v.x_new, cb, pb);
            pose_factor(pa, pa + 3, pb, pb + 3, v.fac_meas + 6 * (size_t)k, v.fac_sqrt + 6 * (size_t)k, r, nullptr);
#pragma unroll
            for (int i = 0; i < 6; ++i) fnew += r[i] * r[i];
            const float* da = v.cam_dir + (size_t)ca * CD_STRIDE;
            const float* db = v.cam_dir + (size_t)cb * CD_STRIDE;
            const float xs[12] = {da[CD_PHI], da[CD_PHI + 1], da[CD_PHI + 2], da[CD_T], da[CD_T + 1], da[CD_T + 2],
                                  db[CD_PHI], db[CD_PHI + 1], db[CD_PHI + 2], db[CD_T], db[CD_T + 1], db[CD_T + 2]};
            const float* Jf = v.fac_J + 72 * (size_t)k;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double t = 0.0;
#pragma unroll
                for (int j = 0; j < 12; ++j) t += (double)Jf[12 * i + j] * (double)xs[j];
                jh2 += t * t;
            }
        }
    }
    double in[2] = {fnew, jh2}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_FACEV], out) && threadIdx.x == 0) {
        st->fac_cost_new = 0.5 * out[0];
        st->fac_jh2 = out[1];
    }
}

// The pose factors' part of the multi-kernel normal operator, after k_matvec in the
// same PCG step (the camera direction records of k_cam_direction, the same camera
// accumulators): J_f^T J_f p into the camera sums, |J_f p|^2 into the matvec slot sums.
__global__ void k_factor_matvec(Views<float> v, const int32_t* gate, const float* zs, int use_beta) {
    (void)zs;
    (void)use_beta;
    if (gated_off(gate)) return;
    __shared__ double red[32];
    DevState* st = v.st;
    float jp2 = 0.0f;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < v.n_fac; k += gridDim.x * blockDim.x) {
        const uint32_t ca = v.fac_cam[2 * (size_t)k], cb = v.fac_cam[2 * (size_t)k + 1];
        jp2 += factor_normal(v.fac_J + 72 * (size_t)k, v.cam_dir + (size_t)ca * CD_STRIDE,
                             v.cam_dir + (size_t)cb * CD_STRIDE, v.cam_acc + (size_t)ca * CA_STRIDE,
                             v.cam_acc + (size_t)cb * CA_STRIDE);
    }
    const double bj = block_sum((double)jp2, red);
    if (threadIdx.x == 0) slot_add(st->acc_mv, 0, bj);
}

void launch_factor_matvec(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                          const float* zs, int use_beta) {
    if (v.n_fac <= 0) return;
    const int grid = std::min(L.item_grid, (v.n_fac + 127) / 128);
    k_factor_matvec<<<grid, 128, 0, s>>>(v, gate, zs, use_beta);
}

void launch_factor_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode) {
    if (v.n_fac <= 0) return;
    const int grid = std::min(L.item_grid, (v.n_fac + 127) / 128);
    k_factor_linearize<<<grid, 128, 0, s>>>(v, mode);
}

void launch_factor_eval(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    if (v.n_fac <= 0) return;
    const int grid = std::min(L.item_grid, (v.n_fac + 127) / 128);
    k_factor_eval<<<grid, 128, 0, s>>>(v);
}

}  // namespace gbba
