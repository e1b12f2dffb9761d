// ba.cu -- one Levenberg-Marquardt step of the tracker's dense visual-inertial
// bundle adjustment (Sec. 3.2: vision residual Eq. 2 over the edges of the frame
// graph, optionally the inertial residual Eq. 3 between consecutive keyframes,
// normal equations solved by the Schur complement of the diagonal depth block,
// Eq. 4).
//
//   r = u*_ij - Pi(T_j T_i^-1 Pi^-1(u, d_i(u)))  for every edge (i, j) and pixel u
//   of keyframe i; cost sum w r^2.  Variables: left perturbations xi_k = (rho, phi)
//   of the poses k >= n_fixed (T_k <- Exp(xi_k) T_k) and every inverse depth.
//   With p = R_ij xbar + d t_ij (the point times its inverse depth):
//     dp/d rho_j = d I, dp/d phi_j = -[p]x,  dp/d rho_i = -d R_ij,
//     dp/d phi_i = R_ij [xbar]x,  dp/d d = t_ij.
//   H = [B E; E^T C] with C diagonal (a residual depends on one inverse depth);
//   (B + damping - E C'^-1 E^T) dxi = -g_xi + E C'^-1 g_d,
//   dd = C'^-1 (-g_d - E^T dxi),  C' = (1 + lambda) C + eps.
//
// Kernels:
//   k_ba_terms  : each thread takes 4 pixels of one edge (i, j): residual and
//                 Jacobians; the 91 values of B_ii, B_ij, B_jj, g_i, g_j and the
//                 cost are reduced per CTA into dense buffers; a 16-float record
//                 per (edge, pixel) keeps E(e, p) = [J_i^T W J_d, J_j^T W J_d] and
//                 the pixel's share of C and g_d.
//   k_ba_schur  : one CTA per (source keyframe i, chunk of pixels): per pixel the
//                 column v_p of E over the slots [pose i, target of each edge out
//                 of i] (summed over the edges for pose i), C'_p and g_d,p from the
//                 records; sum_p v_p v_p^T / C'_p in 2 x 2 register tiles and
//                 sum_p v_p g_d,p / C'_p, added once per CTA into the reduced system.
//   k_ba_inertial: one CTA per consecutive keyframe pair: the 15 residuals of
//                 Eq. 3 and their Jacobian, added into the 15-wide keyframe blocks.
//   k_ba_solve_cluster: a cluster of 8 CTAs: damping, then block Gauss-Jordan
//                 elimination of the symmetric positive definite reduced system
//                 (no pivoting; 6-wide panels read across the cluster through
//                 distributed shared memory; one cluster barrier per panel).
//   k_ba_update : inverse depths by back-substitution, poses by Exp (velocities
//                 and biases added).
#include <cooperative_groups.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kTermThreads = 128;
constexpr int kTermPix = 4;                            // pixels per thread
constexpr int kTermVals = 21 + 36 + 21 + 6 + 6 + 1;   // H_ii (upper), H_ij, H_jj (upper), g_i, g_j, cost
constexpr int kRec = 16;                               // record: E_i (6), E_j (6), C share, g_d share, 2 unused
constexpr int kMaxOut = 15;                            // edges with one source keyframe
constexpr int kMaxSlots = 6 * (1 + kMaxOut);

struct BaDev {
    float* poses;          // [K][12]
    float* disp;           // [K][P]
    const float* targets;  // [E][P][2]
    const float* weights;  // [E][P][2]
    const int32_t* ii;
    const int32_t* jj;
    int K, E, h, w, P, n_fixed, n;   // n = bs (K - n_fixed)
    int bs;                          // variables per free keyframe: 6 (pose), 15 with the inertial factor
    const float* imu;                // [K - 1][GS_BA_IMU_FLOATS] or null
    float* vel;                      // [K][3]
    float* bias;                     // [K][6]
    const float* bias_hat;           // [K][6]
    float gx, gy, gz;                // gravity (world)
    float fx, fy, cx, cy;
    float* rec;            // [E][P][kRec]
    float* SB;             // [n][n] B (undamped)
    float* SS;             // [n][n] -E C'^-1 E^T
    float* rhs;            // [n]
    float* dxi;            // [n]
    float* cost;           // [1]
    int* status;
};

__device__ __forceinline__ bool edge_ok(const BaDev& b, int i, int j) {
    return i >= 0 && i < b.K && j >= 0 && j < b.K && i != j;
}

__device__ __forceinline__ void rel_pose(const BaDev& b, int i, int j, float* Rij, float* tij) {
    const float* Pi = b.poses + 12 * i;
    const float* Pj = b.poses + 12 * j;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            Rij[3 * r + c] = Pj[3 * r] * Pi[3 * c] + Pj[3 * r + 1] * Pi[3 * c + 1] + Pj[3 * r + 2] * Pi[3 * c + 2];
    for (int r = 0; r < 3; r++)
        tij[r] = Pj[9 + r] - (Rij[3 * r] * Pi[9] + Rij[3 * r + 1] * Pi[10] + Rij[3 * r + 2] * Pi[11]);
}

// sum over the CTA of kTermVals values per thread; thread t < kTermVals gets
// total t.  Every thread writes its values as a column of s_all; thread t then
// sums row t (rows padded to an odd length: both passes are free of bank
// conflicts).
__device__ __forceinline__ float block_sum_vals(const float (&v)[kTermVals], float (*s_all)[kTermThreads + 1]) {
#pragma unroll
    for (int k = 0; k < kTermVals; k++) s_all[k][threadIdx.x] = v[k];
    __syncthreads();
    float tot = 0.f;
    if ((int)threadIdx.x < kTermVals) {
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll 8
        for (int j = 0; j < kTermThreads; j += 4) {
            p0 += s_all[threadIdx.x][j];
            p1 += s_all[threadIdx.x][j + 1];
            p2 += s_all[threadIdx.x][j + 2];
            p3 += s_all[threadIdx.x][j + 3];
        }
        tot = (p0 + p1) + (p2 + p3);
    }
    return tot;
}

__global__ void __launch_bounds__(kTermThreads) k_ba_terms(BaDev b) {
    __shared__ float s_all[kTermVals][kTermThreads + 1];
    const int e = blockIdx.y;
    const int i = b.ii[e], j = b.jj[e];
    float v[kTermVals];
#pragma unroll
    for (int k = 0; k < kTermVals; k++) v[k] = 0.f;
    if (!edge_ok(b, i, j)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(b.status, 0, GS_ERR_INVALID_ARG);
        return;   // the whole CTA returns: no barrier is reached
    }
    float Rij[9], tij[3];
    rel_pose(b, i, j, Rij, tij);
    const bool fi = i >= b.n_fixed, fj = j >= b.n_fixed;
    for (int pk = 0; pk < kTermPix; pk++) {
        const int q = ((int)blockIdx.x * kTermPix + pk) * kTermThreads + (int)threadIdx.x;
        if (q >= b.P) break;
        const int y = q / b.w, x = q % b.w;
        const float xb[3] = {((float)x + 0.5f - b.cx) / b.fx, ((float)y + 0.5f - b.cy) / b.fy, 1.0f};
        const float d = b.disp[(size_t)i * b.P + q];
        float p[3];
        for (int r = 0; r < 3; r++) p[r] = Rij[3 * r] * xb[0] + Rij[3 * r + 1] * xb[1] + Rij[3 * r + 2] * xb[2] + d * tij[r];
        const float iz = 1.0f / p[2];
        const size_t o = ((size_t)e * b.P + q) * 2;
        const float r0 = b.targets[o] - (b.fx * p[0] * iz + b.cx);
        const float r1 = b.targets[o + 1] - (b.fy * p[1] * iz + b.cy);
        const float w0 = b.weights[o], w1 = b.weights[o + 1];
        // dr/dp = -dPi/dp
        const float a00 = -b.fx * iz, a02 = b.fx * p[0] * iz * iz;
        const float a11 = -b.fy * iz, a12 = b.fy * p[1] * iz * iz;
        // dp/d(xi_j) = [d I, -[p]x], dp/d(xi_i) = [-d R_ij, R_ij [xb]x]
        float Dj[3][6], Di[3][6];
        const float pk3[3][3] = {{0.f, p[2], -p[1]}, {-p[2], 0.f, p[0]}, {p[1], -p[0], 0.f}};      // -[p]x
        const float xk[3][3] = {{0.f, -xb[2], xb[1]}, {xb[2], 0.f, -xb[0]}, {-xb[1], xb[0], 0.f}}; // [xb]x
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                Dj[r][c] = r == c ? d : 0.f;
                Dj[r][3 + c] = pk3[r][c];
                Di[r][c] = -d * Rij[3 * r + c];
                Di[r][3 + c] = Rij[3 * r] * xk[0][c] + Rij[3 * r + 1] * xk[1][c] + Rij[3 * r + 2] * xk[2][c];
            }
        float Ji[2][6], Jj[2][6];
        for (int c = 0; c < 6; c++) {
            Ji[0][c] = fi ? a00 * Di[0][c] + a02 * Di[2][c] : 0.f;
            Ji[1][c] = fi ? a11 * Di[1][c] + a12 * Di[2][c] : 0.f;
            Jj[0][c] = fj ? a00 * Dj[0][c] + a02 * Dj[2][c] : 0.f;
            Jj[1][c] = fj ? a11 * Dj[1][c] + a12 * Dj[2][c] : 0.f;
        }
        const float Jd0 = a00 * tij[0] + a02 * tij[2], Jd1 = a11 * tij[1] + a12 * tij[2];
        int k = 0;
        for (int a = 0; a < 6; a++)
            for (int c = a; c < 6; c++) v[k++] += w0 * Ji[0][a] * Ji[0][c] + w1 * Ji[1][a] * Ji[1][c];
        for (int a = 0; a < 6; a++)
            for (int c = 0; c < 6; c++) v[k++] += w0 * Ji[0][a] * Jj[0][c] + w1 * Ji[1][a] * Jj[1][c];
        for (int a = 0; a < 6; a++)
            for (int c = a; c < 6; c++) v[k++] += w0 * Jj[0][a] * Jj[0][c] + w1 * Jj[1][a] * Jj[1][c];
        for (int a = 0; a < 6; a++) v[k++] += w0 * Ji[0][a] * r0 + w1 * Ji[1][a] * r1;
        for (int a = 0; a < 6; a++) v[k++] += w0 * Jj[0][a] * r0 + w1 * Jj[1][a] * r1;
        v[k] += w0 * r0 * r0 + w1 * r1 * r1;
        float rc[kRec];
        for (int a = 0; a < 6; a++) {
            rc[a] = w0 * Ji[0][a] * Jd0 + w1 * Ji[1][a] * Jd1;
            rc[6 + a] = w0 * Jj[0][a] * Jd0 + w1 * Jj[1][a] * Jd1;
        }
        rc[12] = w0 * Jd0 * Jd0 + w1 * Jd1 * Jd1;
        rc[13] = w0 * Jd0 * r0 + w1 * Jd1 * r1;
        rc[14] = 0.f;
        rc[15] = 0.f;
        float4* ro = reinterpret_cast<float4*>(b.rec + ((size_t)e * b.P + q) * kRec);
#pragma unroll
        for (int m = 0; m < kRec / 4; m++) ro[m] = make_float4(rc[4 * m], rc[4 * m + 1], rc[4 * m + 2], rc[4 * m + 3]);
    }
    const float tot = block_sum_vals(v, s_all);
    const int t = threadIdx.x;
    if (t < kTermVals) {
        const int bi = b.bs * (i - b.n_fixed), bj = b.bs * (j - b.n_fixed);
        if (t < 21) {
            if (i >= b.n_fixed) {
                int a = 0, c = t, rem = t;          // t -> (a, c), c >= a
                while (rem >= 6 - a) { rem -= 6 - a; a++; }
                c = a + rem;
                atomicAdd(b.SB + (size_t)(bi + a) * b.n + bi + c, tot);
                if (c != a) atomicAdd(b.SB + (size_t)(bi + c) * b.n + bi + a, tot);
            }
        } else if (t < 57) {
            if (i >= b.n_fixed && j >= b.n_fixed) {
                const int a = (t - 21) / 6, c = (t - 21) % 6;
                atomicAdd(b.SB + (size_t)(bi + a) * b.n + bj + c, tot);
                atomicAdd(b.SB + (size_t)(bj + c) * b.n + bi + a, tot);
            }
        } else if (t < 78) {
            if (j >= b.n_fixed) {
                int a = 0, rem = t - 57;
                while (rem >= 6 - a) { rem -= 6 - a; a++; }
                const int c = a + rem;
                atomicAdd(b.SB + (size_t)(bj + a) * b.n + bj + c, tot);
                if (c != a) atomicAdd(b.SB + (size_t)(bj + c) * b.n + bj + a, tot);
            }
        } else if (t < 84) {
            if (i >= b.n_fixed) atomicAdd(b.rhs + bi + (t - 78), -tot);
        } else if (t < 90) {
            if (j >= b.n_fixed) atomicAdd(b.rhs + bj + (t - 84), -tot);
        } else {
            atomicAdd(b.cost, tot);
        }
    }
}

// ------------------------------------------------------------ inertial factor
// Eq. 3 between consecutive keyframes i, j = i + 1, on the body-to-world rotation
// R_i = R_cw,i^T, position p_i = -R_i t_cw,i, velocity v_i and bias b_i = (b_g, b_a)
// (the camera frame taken as the body frame).  Under the perturbation of the
// visual part (T_cw <- Exp(xi) T_cw, xi = (rho, phi)) R_i <- R_i Exp(-phi) and
// p_i <- p_i - R_i rho to first order; v and b are additive.  With E = R_i^T R_j,
// A = dR Exp(J_rot db_g), M = A^T E, r_rot = Log(M), J_r the right Jacobian of
// SO(3) and Jri = J_r(r_rot)^-1:
//   d r_rot / d phi_i = Jri M^T A^T,  d r_rot / d phi_j = -Jri,
//   d r_rot / d b_g,i = -Jri M^T J_r(J_rot db_g) J_rot,
//   r_pos = q - (dp + J_pos db), q = R_i^T (p_j - p_i - v_i dt - g dt^2 / 2):
//     d / d rho_i = I, d / d phi_i = -[q]x, d / d rho_j = -E, d / d v_i = -R_i^T dt,
//     d / d b_i = -J_pos,
//   r_vel = q' - (dv + J_vel db), q' = R_i^T (v_j - v_i - g dt):
//     d / d phi_i = -[q']x, d / d v_i = -R_i^T, d / d v_j = R_i^T, d / d b_i = -J_vel,
//   r_bias = b_j - b_i.
// Keyframe variables (15): rho 0-2, phi 3-5, v 6-8, b_g 9-11, b_a 12-14.

__device__ __forceinline__ void skew3(const float* w, float* K) {
    K[0] = 0.f;   K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2];  K[4] = 0.f;   K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0];  K[8] = 0.f;
}
__device__ __forceinline__ void mat3mul(const float* A, const float* B, float* C) {     // C = A B
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}
__device__ __forceinline__ void mat3tmul(const float* A, const float* B, float* C) {    // C = A^T B
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[3 * r + c] = A[r] * B[c] + A[3 + r] * B[3 + c] + A[6 + r] * B[6 + c];
}
// I + a K + b K^2 for K = [w]x
__device__ __forceinline__ void so3_poly(const float* w, float a, float bcoef, float* M) {
    float K[9], K2[9];
    skew3(w, K);
    mat3mul(K, K, K2);
    for (int k = 0; k < 9; k++) M[k] = (k % 4 == 0 ? 1.f : 0.f) + a * K[k] + bcoef * K2[k];
}
__device__ __forceinline__ void so3_exp_f(const float* w, float* M) {
    const float th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = sqrtf(th2);
    const float a = th < 1e-4f ? 1.f - th2 / 6.f : sinf(th) / th;
    const float bc = th < 1e-4f ? 0.5f - th2 / 24.f : (1.f - cosf(th)) / th2;
    so3_poly(w, a, bc, M);
}
__device__ __forceinline__ void so3_log_f(const float* M, float* w) {
    const float c = fminf(1.f, fmaxf(-1.f, 0.5f * (M[0] + M[4] + M[8] - 1.f)));
    const float th = acosf(c);
    const float f = th < 1e-4f ? 0.5f * (1.f + th * th / 6.f) : 0.5f * th / sinf(th);
    w[0] = f * (M[7] - M[5]); w[1] = f * (M[2] - M[6]); w[2] = f * (M[3] - M[1]);
}
// right Jacobian J_r(x) = I - (1 - cos t) / t^2 [x]x + (t - sin t) / t^3 [x]x^2
__device__ __forceinline__ void so3_jr(const float* x, float* J) {
    const float th2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2], th = sqrtf(th2);
    const float a = th < 1e-3f ? 0.5f - th2 / 24.f : (1.f - cosf(th)) / th2;
    const float bc = th < 1e-3f ? 1.f / 6.f - th2 / 120.f : (th - sinf(th)) / (th2 * th);
    so3_poly(x, -a, bc, J);
}
// its inverse: I + [r]x / 2 + (1 / t^2 - (1 + cos t) / (2 t sin t)) [r]x^2
__device__ __forceinline__ void so3_jr_inv(const float* r, float* J) {
    const float th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], th = sqrtf(th2);
    const float bc = th < 1e-3f ? 1.f / 12.f + th2 / 720.f : 1.f / th2 - (1.f + cosf(th)) / (2.f * th * sinf(th));
    so3_poly(r, 0.5f, bc, J);
}

constexpr int kImuFloats = GS_BA_IMU_FLOATS;
constexpr int kInerThreads = 256;

// One CTA per consecutive pair (i, i + 1): thread 0 forms the residual r (15) and
// the Jacobian J (15 x 30) in shared memory; then H += J^T W J, rhs -= J^T W r and
// the cost += r^T W r over the free keyframes' blocks.
__global__ void __launch_bounds__(kInerThreads) k_ba_inertial(BaDev b) {
    __shared__ float sJ[15][30], sWJ[15][30], sW[15][15], sr[15], sWr[15];
    const int i = blockIdx.x, j = i + 1, t = threadIdx.x;
    const float* rec = b.imu + (size_t)i * kImuFloats;
    for (int k = t; k < 225; k += kInerThreads) sW[k / 15][k % 15] = rec[61 + k];
    for (int k = t; k < 450; k += kInerThreads) sJ[k / 30][k % 30] = 0.f;
    __syncthreads();
    if (t == 0) {
        const float* dR = rec;
        const float* dp = rec + 9;
        const float* dv = rec + 12;
        const float* Jrot = rec + 15;
        const float* Jpos = rec + 24;        // 3 x 6
        const float* Jvel = rec + 42;        // 3 x 6
        const float dt = rec[60];
        // body-to-world rotations and positions from the world-to-camera poses
        const float* Pi = b.poses + 12 * i;
        const float* Pj = b.poses + 12 * j;
        float Ri[9], Rj[9], pi_[3], pj_[3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) { Ri[3 * r + c] = Pi[3 * c + r]; Rj[3 * r + c] = Pj[3 * c + r]; }
        for (int r = 0; r < 3; r++) {
            pi_[r] = -(Ri[3 * r] * Pi[9] + Ri[3 * r + 1] * Pi[10] + Ri[3 * r + 2] * Pi[11]);
            pj_[r] = -(Rj[3 * r] * Pj[9] + Rj[3 * r + 1] * Pj[10] + Rj[3 * r + 2] * Pj[11]);
        }
        const float* vi = b.vel + 3 * i;
        const float* vj = b.vel + 3 * j;
        const float* bi = b.bias + 6 * i;
        const float* bj = b.bias + 6 * j;
        float db[6];
        for (int k = 0; k < 6; k++) db[k] = bi[k] - b.bias_hat[6 * i + k];
        const float g[3] = {b.gx, b.gy, b.gz};
        // rotation
        float jd[3], Ej[9], A[9], E[9], M[9], rr[3], Jri[9];
        for (int r = 0; r < 3; r++) jd[r] = Jrot[3 * r] * db[0] + Jrot[3 * r + 1] * db[1] + Jrot[3 * r + 2] * db[2];
        so3_exp_f(jd, Ej);
        mat3mul(dR, Ej, A);
        mat3tmul(Ri, Rj, E);
        mat3tmul(A, E, M);
        so3_log_f(M, rr);
        so3_jr_inv(rr, Jri);
        float MtAt[9], T1[9], Jrd[9], T2[9];
        {
            float AM[9];
            mat3mul(A, M, AM);                          // (A M)^T = M^T A^T
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) MtAt[3 * r + c] = AM[3 * c + r];
        }
        mat3mul(Jri, MtAt, T1);                         // d r_rot / d phi_i
        so3_jr(jd, Jrd);
        {
            float JrdJrot[9], Mt[9];
            mat3mul(Jrd, Jrot, JrdJrot);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) Mt[3 * r + c] = M[3 * c + r];
            float MtJ[9];
            mat3mul(Mt, JrdJrot, MtJ);
            mat3mul(Jri, MtJ, T2);                      // -(d r_rot / d b_g,i)
        }
        for (int r = 0; r < 3; r++) {
            sr[r] = rr[r];
            for (int c = 0; c < 3; c++) {
                sJ[r][3 + c] = T1[3 * r + c];
                sJ[r][15 + 3 + c] = -Jri[3 * r + c];
                sJ[r][9 + c] = -T2[3 * r + c];
            }
        }
        // position and velocity
        float sp[3], sv[3], q[3], qv[3];
        for (int r = 0; r < 3; r++) {
            sp[r] = pj_[r] - pi_[r] - vi[r] * dt - 0.5f * g[r] * dt * dt;
            sv[r] = vj[r] - vi[r] - g[r] * dt;
        }
        for (int r = 0; r < 3; r++) {
            q[r] = Ri[r] * sp[0] + Ri[3 + r] * sp[1] + Ri[6 + r] * sp[2];
            qv[r] = Ri[r] * sv[0] + Ri[3 + r] * sv[1] + Ri[6 + r] * sv[2];
        }
        float Kq[9], Kqv[9];
        skew3(q, Kq);
        skew3(qv, Kqv);
        for (int r = 0; r < 3; r++) {
            float cp = 0.f, cv = 0.f;
            for (int k = 0; k < 6; k++) { cp += Jpos[6 * r + k] * db[k]; cv += Jvel[6 * r + k] * db[k]; }
            sr[3 + r] = q[r] - (dp[r] + cp);
            sr[6 + r] = qv[r] - (dv[r] + cv);
            for (int c = 0; c < 3; c++) {
                sJ[3 + r][c] = r == c ? 1.f : 0.f;                      // rho_i
                sJ[3 + r][3 + c] = -Kq[3 * r + c];                      // phi_i
                sJ[3 + r][15 + c] = -E[3 * r + c];                      // rho_j
                sJ[3 + r][6 + c] = -Ri[3 * c + r] * dt;                  // v_i
                sJ[6 + r][3 + c] = -Kqv[3 * r + c];                     // phi_i
                sJ[6 + r][6 + c] = -Ri[3 * c + r];                      // v_i
                sJ[6 + r][15 + 6 + c] = Ri[3 * c + r];                  // v_j
            }
            for (int k = 0; k < 6; k++) {
                sJ[3 + r][9 + k] = -Jpos[6 * r + k];
                sJ[6 + r][9 + k] = -Jvel[6 * r + k];
            }
        }
        // bias smoothness
        for (int k = 0; k < 6; k++) {
            sr[9 + k] = bj[k] - bi[k];
            sJ[9 + k][9 + k] = -1.f;
            sJ[9 + k][15 + 9 + k] = 1.f;
        }
    }
    __syncthreads();
    // W J and W r
    for (int k = t; k < 15 * 30 + 15; k += kInerThreads) {
        const int r = k < 450 ? k / 30 : k - 450, c = k < 450 ? k % 30 : 0;
        float acc = 0.f;
        for (int m = 0; m < 15; m++) acc += sW[r][m] * (k < 450 ? sJ[m][c] : sr[m]);
        if (k < 450) sWJ[r][c] = acc;
        else sWr[r] = acc;
    }
    __syncthreads();
    // J^T W J into the free blocks, J^T W r into the right-hand side, r^T W r into the cost
    auto row_of = [&](int c) {
        const int kf = c < 15 ? i : j;
        return kf >= b.n_fixed ? b.bs * (kf - b.n_fixed) + c % 15 : -1;
    };
    for (int k = t; k < 30 * 30; k += kInerThreads) {
        const int a = k / 30, c = k % 30;
        const int ra = row_of(a), rc = row_of(c);
        if (ra < 0 || rc < 0) continue;
        float acc = 0.f;
        for (int m = 0; m < 15; m++) acc += sJ[m][a] * sWJ[m][c];
        atomicAdd(b.SB + (size_t)ra * b.n + rc, acc);
    }
    if (t < 30) {
        const int ra = row_of(t);
        if (ra >= 0) {
            float acc = 0.f;
            for (int m = 0; m < 15; m++) acc += sJ[m][t] * sWr[m];
            atomicAdd(b.rhs + ra, -acc);
        }
    } else if (t == 32) {
        float acc = 0.f;
        for (int m = 0; m < 15; m++) acc += sr[m] * sWr[m];
        atomicAdd(b.cost, acc);
    }
}

// The edges out of keyframe i (valid ones, in edge order) into s_out[0 .. kMaxOut);
// *s_deg = their count (which may exceed kMaxOut).  Called by every thread of
// the CTA; ends with a barrier.
__device__ __forceinline__ void out_edges(const BaDev& b, int i, int* s_out, int* s_deg) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int deg = 0;
        for (int e0 = 0; e0 < b.E; e0 += 32) {
            const int e = e0 + lane;
            const bool is = e < b.E && b.ii[e] == i && edge_ok(b, i, b.jj[e]);
            const uint32_t m = __ballot_sync(0xffffffffu, is);
            if (is) {
                const int pos = deg + __popc(m & ((1u << lane) - 1u));
                if (pos < kMaxOut) s_out[pos] = e;
            }
            deg += __popc(m);
        }
        if (lane == 0) *s_deg = deg;
    }
    __syncthreads();
}

// Schur complement of the inverse-depth block.  CTA (chunk, i): the pixels
// [chunk * kSchurChunk, ...) of source keyframe i.  Slot 0 is pose i, slot 1 + k
// the target of the k-th edge out of i; v_p (6 per slot, m = 6 (1 + deg) rows) is
// the column of E of pixel p's inverse depth.  Row m of the staged block holds
// g_d,p and row m + 1 zeros, so the 2 x 2 register tiles of the upper triangle of
// sum_p u_p [v_p; g_d,p; 0]^T (u_p = v_p / C'_p) give both E C'^-1 E^T and, in
// their last column, E C'^-1 g_d.
constexpr int kSchurThreads = 256;
constexpr int kSchurPix = 32;            // pixels staged per round
constexpr int kSchurChunk = 256;         // pixels per CTA
constexpr int kSchurRows = kMaxSlots + 2;
constexpr int kMaxTileRows = kSchurRows / 2;
constexpr int kTilesPerThread = (kMaxTileRows * (kMaxTileRows + 1) / 2 + kSchurThreads - 1) / kSchurThreads;
static_assert(kSchurPix * 8 == kSchurThreads, "one (pixel, record float pair) per thread");

__global__ void __launch_bounds__(kSchurThreads) k_ba_schur(BaDev b, float lambda, float eps) {
    __shared__ int s_out[kMaxOut];
    __shared__ int s_deg;
    // rows padded by 4 floats: 2 x 2 tiles of one warp read rows at different
    // bank offsets instead of all starting at bank 0
    __shared__ __align__(16) float s_v[kSchurRows][kSchurPix + 4];
    __shared__ __align__(16) float s_u[kSchurRows][kSchurPix + 4];
    __shared__ float s_w[kSchurPix];
    const int i = blockIdx.y, t = threadIdx.x;
    out_edges(b, i, s_out, &s_deg);
    const int deg = s_deg;
    if (deg == 0) return;
    if (deg > kMaxOut) {
        if (t == 0 && blockIdx.x == 0) atomicCAS(b.status, 0, GS_ERR_UNSUPPORTED);
        return;
    }
    const int m = 6 * (1 + deg), T = m / 2 + 1, n_tiles = T * (T + 1) / 2;
    int ta[kTilesPerThread], tb[kTilesPerThread];
    float acc[kTilesPerThread][4];
#pragma unroll
    for (int s = 0; s < kTilesPerThread; s++) {
        int rem = t + s * kSchurThreads, a = 0;
        if (rem < n_tiles) {
            while (rem >= T - a) { rem -= T - a; a++; }
            ta[s] = a; tb[s] = a + rem;
        } else {
            ta[s] = -1; tb[s] = -1;
        }
        acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.f;
    }
    // this thread's pixel and pair of record floats: pairs 0-2 are E_i (summed over
    // the edges into slot 0), 3-5 E_j (slot 1 + k), 6 the C and g_d shares (summed)
    const int spx = t / 8, f8 = t % 8;
    if (t < kSchurPix) s_v[m + 1][t] = 0.f;      // row m is rewritten every round
    const int p_lo = blockIdx.x * kSchurChunk, p_hi = min(b.P, p_lo + kSchurChunk);
    for (int p0 = p_lo; p0 < p_hi; p0 += kSchurPix) {
        const bool px_ok = spx < p_hi - p0;
        // all of the round's loads are issued before the first store
        float2 rv[kMaxOut];
#pragma unroll
        for (int k = 0; k < kMaxOut; k++) {
            const bool ok = k < deg && px_ok && f8 < 7;
            rv[k] = ok ? *reinterpret_cast<const float2*>(b.rec + ((size_t)s_out[ok ? k : 0] * b.P + p0 + spx) * kRec +
                                                          2 * f8)
                       : make_float2(0.f, 0.f);
        }
        if (f8 < 3 || f8 == 6) {
            float2 sum = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kMaxOut; k++) { sum.x += rv[k].x; sum.y += rv[k].y; }
            if (f8 < 3) {
                s_v[2 * f8][spx] = sum.x;
                s_v[2 * f8 + 1][spx] = sum.y;
            } else {
                s_w[spx] = px_ok ? 1.0f / ((1.0f + lambda) * sum.x + eps) : 0.f;
                s_v[m][spx] = sum.y;
            }
        } else if (f8 < 6) {
#pragma unroll
            for (int k = 0; k < kMaxOut; k++) {
                if (k < deg) {
                    s_v[6 + 6 * k + 2 * (f8 - 3)][spx] = rv[k].x;
                    s_v[6 + 6 * k + 2 * (f8 - 3) + 1][spx] = rv[k].y;
                }
            }
        }
        __syncthreads();
        for (int idx = t; idx < m * kSchurPix; idx += kSchurThreads) {
            const int a = idx / kSchurPix, px = idx % kSchurPix;
            s_u[a][px] = s_v[a][px] * s_w[px];
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < kTilesPerThread; s++) {
            if (ta[s] < 0 || 2 * ta[s] >= m) continue;     // rows m, m + 1 of u are not needed
            const float4* u0 = reinterpret_cast<const float4*>(s_u[2 * ta[s]]);
            const float4* u1 = reinterpret_cast<const float4*>(s_u[2 * ta[s] + 1]);
            const float4* v0 = reinterpret_cast<const float4*>(s_v[2 * tb[s]]);
            const float4* v1 = reinterpret_cast<const float4*>(s_v[2 * tb[s] + 1]);
#pragma unroll
            for (int q = 0; q < kSchurPix / 4; q++) {
                const float4 a0 = u0[q], a1 = u1[q], c0 = v0[q], c1 = v1[q];
                acc[s][0] += a0.x * c0.x + a0.y * c0.y + a0.z * c0.z + a0.w * c0.w;
                acc[s][1] += a0.x * c1.x + a0.y * c1.y + a0.z * c1.z + a0.w * c1.w;
                acc[s][2] += a1.x * c0.x + a1.y * c0.y + a1.z * c0.z + a1.w * c0.w;
                acc[s][3] += a1.x * c1.x + a1.y * c1.y + a1.z * c1.z + a1.w * c1.w;
            }
        }
        __syncthreads();
    }
    auto slot_pose = [&](int slot) { return slot == 0 ? i : b.jj[s_out[slot - 1]]; };
#pragma unroll
    for (int s = 0; s < kTilesPerThread; s++) {
        if (ta[s] < 0 || 2 * ta[s] >= m) continue;
#pragma unroll
        for (int xy = 0; xy < 4; xy++) {
            const int a = 2 * ta[s] + (xy >> 1), c = 2 * tb[s] + (xy & 1);
            if (a > c || c == m + 1) continue;         // the lower element of a diagonal tile; the zero row
            const int pa = slot_pose(a / 6);
            if (pa < b.n_fixed) continue;
            const int ra = b.bs * (pa - b.n_fixed) + a % 6;
            if (c == m) {                               // E C'^-1 g_d
                atomicAdd(b.rhs + ra, acc[s][xy]);
                continue;
            }
            const int pc = slot_pose(c / 6);
            if (pc < b.n_fixed) continue;
            const int rc = b.bs * (pc - b.n_fixed) + c % 6;
            atomicAdd(b.SS + (size_t)ra * b.n + rc, -acc[s][xy]);
            if (a != c) atomicAdd(b.SS + (size_t)rc * b.n + ra, -acc[s][xy]);
        }
    }
}

// Solve of the reduced system (B damped - E C'^-1 E^T) dxi = rhs in 6 x 6 pose
// panels (a system that is not a multiple of 6 is padded with identity rows).
constexpr int kNb = 6;

// LU of a 6 x 6 block in registers: unit-lower multipliers below the diagonal,
// U on and above it; inv[k] = 1 / U_kk.
__device__ __forceinline__ void lu6(float (&a)[kNb][kNb], float (&inv)[kNb]) {
#pragma unroll
    for (int k = 0; k < kNb; k++) {
        inv[k] = __frcp_rn(fmaxf(a[k][k], 1e-30f));
#pragma unroll
        for (int r = k + 1; r < kNb; r++) {
            const float f = a[r][k] * inv[k];
            a[r][k] = f;
#pragma unroll
            for (int c = k + 1; c < kNb; c++) a[r][c] -= f * a[k][c];
        }
    }
}

// ------------------------------------------------------- cluster solve
// The same damped system solved by a cluster of kClusterCtas CTAs with block
// Gauss-Jordan elimination.  CTA q keeps the row panels p = q, q + C, ... in its
// shared memory.  Step k: every CTA copies panel k's rows (columns kb .. n) out of
// the owner's shared memory, forms W = A_kk^-1 A[panel k, k1 ..] (one column per
// thread, the 6 x 6 factorisation redundantly in registers) and eliminates the
// panel's columns from all of its own rows above and below the panel:
// A[r, k1 ..] -= A[r, panel k] W.  Panel k's rows are not written during step k,
// and a cluster barrier ends every step, so each copy reads finished rows.  After
// the last step the system is block diagonal and each CTA solves its own panels,
// A_pp x_p = rhs_p, with A_pp as it stood at step p (later steps only touch the
// columns to the right of their panel).
namespace cg = cooperative_groups;
constexpr int kClusterCtas = 8;
constexpr int kClSolveThreads = 256;
constexpr int kClWarps = kClSolveThreads / 32;

__host__ __device__ inline int cl_panels(int np, int q) { return (np - q + kClusterCtas - 1) / kClusterCtas; }

template <int CPL>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClSolveThreads)
    k_ba_solve_cluster(BaDev b, float lambda, float eps) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float sm[];
    const int q = (int)cl.block_rank();
    const int n0 = b.n, n = (n0 + kNb - 1) / kNb * kNb, ld = n + 1, np = n / kNb;
    const int mine = cl_panels(np, q), rows = mine * kNb;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    float* R = sm;                                  // [rows][ld] this CTA's rows
    float* P = R + (size_t)rows * ld;               // [6][ld] the current panel's rows
    float* W = P + (size_t)kNb * ld;                // [6][ld] A_kk^-1 A[panel k, k1 ..]
    __shared__ int s_bad;
    // own rows of the damped system; padding rows are identity, padding columns zero
    for (int k = t; k < rows * ld; k += kClSolveThreads) {
        const int lr = k / ld, c = k - lr * ld;
        const int r = kNb * (q + kClusterCtas * (lr / kNb)) + lr % kNb;
        float v;
        if (c == n) {
            v = r < n0 ? b.rhs[r] : 0.f;
        } else if (r < n0 && c < n0) {
            const size_t g = (size_t)r * n0 + c;
            v = b.SS[g] + (r == c ? (1.0f + lambda) * b.SB[g] + eps : b.SB[g]);
        } else {
            v = r == c ? 1.f : 0.f;
        }
        R[k] = v;
    }
    if (t == 0) s_bad = 0;
    cl.sync();
    for (int k = 0; k < np; k++) {
        const int kb = kNb * k, k1 = kb + kNb, owner = k % kClusterCtas, lpk = k / kClusterCtas;
        const int ncols = ld - k1;
        {
            // all remote loads of a thread issued before its stores (wdt <= ld <= 229 < 2 * 256)
            const float* src = cl.map_shared_rank(R, owner) + (size_t)lpk * kNb * ld;
            float v[kNb][2];
#pragma unroll
            for (int m = 0; m < kNb; m++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int c = kb + t + h * kClSolveThreads;
                    v[m][h] = c < ld ? src[(size_t)m * ld + c] : 0.f;
                }
#pragma unroll
            for (int m = 0; m < kNb; m++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int c = kb + t + h * kClSolveThreads;
                    if (c < ld) P[m * ld + c] = v[m][h];
                }
        }
        __syncthreads();
        if (t < ncols || t == 0) {
            float a[kNb][kNb], inv[kNb];
#pragma unroll
            for (int r = 0; r < kNb; r++)
#pragma unroll
                for (int c = 0; c < kNb; c++) a[r][c] = P[r * ld + kb + c];
            lu6(a, inv);
            if (t == 0 && q == owner) {
#pragma unroll
                for (int m = 0; m < kNb; m++)
                    if (!(a[m][m] > 0.f)) s_bad = 1;
            }
            for (int j = t; j < ncols; j += kClSolveThreads) {
                const int c = k1 + j;
                float y[kNb];
#pragma unroll
                for (int m = 0; m < kNb; m++) y[m] = P[m * ld + c];
#pragma unroll
                for (int m = 1; m < kNb; m++)
#pragma unroll
                    for (int u = 0; u < m; u++) y[m] -= a[m][u] * y[u];
#pragma unroll
                for (int m = kNb - 1; m >= 0; m--) {
#pragma unroll
                    for (int u = m + 1; u < kNb; u++) y[m] -= a[m][u] * y[u];
                    y[m] *= inv[m];
                }
#pragma unroll
                for (int m = 0; m < kNb; m++) W[m * ld + c] = y[m];
            }
        }
        __syncthreads();
        if (ncols > 0 && rows > 0) {
            const int jn = (ncols + 31) >> 5;
            float w[CPL][kNb];
#pragma unroll
            for (int j = 0; j < CPL; j++) {
                const int c = k1 + lane + 32 * j;
                if (j < jn) {
#pragma unroll
                    for (int m = 0; m < kNb; m++) w[j][m] = c < ld ? W[m * ld + c] : 0.f;
                }
            }
            for (int lr = warp; lr < rows; lr += kClWarps) {
                if (q == owner && lr / kNb == lpk) continue;      // the panel's own rows (warp-uniform)
                float* row = R + (size_t)lr * ld;
                float l[kNb];
#pragma unroll
                for (int m = 0; m < kNb; m++) l[m] = row[kb + m];
                float v[CPL];
#pragma unroll
                for (int j = 0; j < CPL; j++) {
                    const int c = k1 + lane + 32 * j;
                    if (j < jn) v[j] = c < ld ? row[c] : 0.f;
                }
#pragma unroll
                for (int j = 0; j < CPL; j++) {
                    if (j < jn) {
#pragma unroll
                        for (int m = 0; m < kNb; m++) v[j] -= l[m] * w[j][m];
                    }
                }
#pragma unroll
                for (int j = 0; j < CPL; j++) {
                    const int c = k1 + lane + 32 * j;
                    if (j < jn && c < ld) row[c] = v[j];
                }
            }
        }
        cl.sync();
    }
    // x_p = A_pp^-1 rhs_p for this CTA's panels
    if (t < mine) {
        const int p = q + kClusterCtas * t, kb = kNb * p;
        const float* rp = R + (size_t)t * kNb * ld;
        float a[kNb][kNb], inv[kNb], y[kNb];
#pragma unroll
        for (int r = 0; r < kNb; r++) {
#pragma unroll
            for (int c = 0; c < kNb; c++) a[r][c] = rp[r * ld + kb + c];
            y[r] = rp[r * ld + n];
        }
        lu6(a, inv);
#pragma unroll
        for (int m = 1; m < kNb; m++)
#pragma unroll
            for (int u = 0; u < m; u++) y[m] -= a[m][u] * y[u];
#pragma unroll
        for (int m = kNb - 1; m >= 0; m--) {
#pragma unroll
            for (int u = m + 1; u < kNb; u++) y[m] -= a[m][u] * y[u];
            y[m] *= inv[m];
        }
#pragma unroll
        for (int m = 0; m < kNb; m++)
            if (kb + m < n0) b.dxi[kb + m] = y[m];
    }
    __syncthreads();
    if (t == 0 && s_bad) atomicCAS(b.status, 0, GS_ERR_NUMERIC);
}

__device__ __forceinline__ float pose_dxi(const BaDev& b, int k, int c) {
    return k >= b.n_fixed ? b.dxi[b.bs * (k - b.n_fixed) + c] : 0.f;
}

// dd_p = C'_p^-1 (-g_d,p - sum_e E(e, p) . [dxi_i, dxi_j]) for every pixel of every
// source keyframe; then the poses T_k <- Exp(dxi_k) T_k (rotation exact,
// translation first order).
constexpr int kUpdateThreads = 256;

__global__ void __launch_bounds__(kUpdateThreads) k_ba_update(BaDev b, float lambda, float eps) {
    __shared__ int s_out[kMaxOut];
    __shared__ int s_deg;
    __shared__ float s_dx[1 + kMaxOut][6];
    const int i = blockIdx.y, t = threadIdx.x;
    out_edges(b, i, s_out, &s_deg);
    const int deg = s_deg;
    if (deg <= kMaxOut && deg > 0) {
        if (t < 6 * (1 + deg)) {
            const int slot = t / 6, c = t % 6;
            s_dx[slot][c] = pose_dxi(b, slot == 0 ? i : b.jj[s_out[slot - 1]], c);
        }
        __syncthreads();
        const int q = blockIdx.x * kUpdateThreads + t;
        if (q < b.P) {
            // the records of four edges in flight at a time
            float C = 0.f, sacc = 0.f;
            for (int k0 = 0; k0 < deg; k0 += 4) {
                float4 rr[4][4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int k = k0 + u;
                    const float4* ro =
                        reinterpret_cast<const float4*>(b.rec + ((size_t)s_out[k < deg ? k : 0] * b.P + q) * kRec);
#pragma unroll
                    for (int h = 0; h < 4; h++) rr[u][h] = k < deg ? ro[h] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int k = k0 + u;
                    if (k >= deg) break;
                    const float4 r0 = rr[u][0], r1 = rr[u][1], r2 = rr[u][2], r3 = rr[u][3];
                    C += r3.x;
                    sacc -= r3.y;
                    sacc -= r0.x * s_dx[0][0] + r0.y * s_dx[0][1] + r0.z * s_dx[0][2] + r0.w * s_dx[0][3] +
                            r1.x * s_dx[0][4] + r1.y * s_dx[0][5];
                    sacc -= r1.z * s_dx[k + 1][0] + r1.w * s_dx[k + 1][1] + r2.x * s_dx[k + 1][2] +
                            r2.y * s_dx[k + 1][3] + r2.z * s_dx[k + 1][4] + r2.w * s_dx[k + 1][5];
                }
            }
            // an inverse depth no residual constrains (all weights 0) keeps its value
            if (C > 0.f) b.disp[(size_t)i * b.P + q] += sacc / ((1.0f + lambda) * C + eps);
        }
    }
    if (blockIdx.x == 0 && t == 0 && i >= b.n_fixed) {
        float rho[3], phi[3];
        for (int c = 0; c < 3; c++) { rho[c] = pose_dxi(b, i, c); phi[c] = pose_dxi(b, i, 3 + c); }
        const float th = sqrtf(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
        const float A = th > 1e-8f ? sinf(th) / th : 1.0f, Bc = th > 1e-8f ? (1.0f - cosf(th)) / (th * th) : 0.5f;
        const float Kx[9] = {0.f, -phi[2], phi[1], phi[2], 0.f, -phi[0], -phi[1], phi[0], 0.f};
        float Rp[9];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                float kk = 0.f;
                for (int m = 0; m < 3; m++) kk += Kx[3 * r + m] * Kx[3 * m + c];
                Rp[3 * r + c] = (r == c ? 1.f : 0.f) + A * Kx[3 * r + c] + Bc * kk;
            }
        if (b.bs == 15) {
            for (int c = 0; c < 3; c++) b.vel[3 * i + c] += b.dxi[15 * (i - b.n_fixed) + 6 + c];
            for (int c = 0; c < 6; c++) b.bias[6 * i + c] += b.dxi[15 * (i - b.n_fixed) + 9 + c];
        }
        // no CTA of this kernel reads the poses (only dxi), so keyframe i's pose can
        // be rewritten here by one thread
        float* P = b.poses + 12 * i;
        float R[9], tt[3];
        for (int m = 0; m < 9; m++) R[m] = P[m];
        for (int m = 0; m < 3; m++) tt[m] = P[9 + m];
        for (int r = 0; r < 3; r++) {
            for (int c = 0; c < 3; c++) P[3 * r + c] = Rp[3 * r] * R[c] + Rp[3 * r + 1] * R[3 + c] + Rp[3 * r + 2] * R[6 + c];
            P[9 + r] = Rp[3 * r] * tt[0] + Rp[3 * r + 1] * tt[1] + Rp[3 * r + 2] * tt[2] + rho[r];
        }
    }
}

}  // namespace

size_t ba_workspace(int K, int E, int P, int n) {
    (void)K;
    return align_up(sizeof(float) * (size_t)E * P * kRec, 256) + 2 * align_up(sizeof(float) * (size_t)n * n, 256) +
           2 * align_up(sizeof(float) * (size_t)(n + 1), 256);
}

cudaError_t launch_ba_step(const gs_ba_problem& pr, float lambda, float eps, float* cost, void* ws,
                           cudaStream_t s) {
    BaDev b;
    b.poses = pr.poses; b.disp = pr.disp; b.targets = pr.targets; b.weights = pr.weights;
    b.ii = pr.ii; b.jj = pr.jj;
    b.K = pr.n_keyframes; b.E = pr.n_edges; b.h = pr.height; b.w = pr.width; b.P = pr.height * pr.width;
    b.n_fixed = pr.n_fixed;
    b.imu = pr.imu; b.vel = pr.vel; b.bias = pr.bias; b.bias_hat = pr.bias_hat;
    b.gx = pr.gravity[0]; b.gy = pr.gravity[1]; b.gz = pr.gravity[2];
    b.bs = pr.imu != nullptr ? 15 : 6;
    b.n = b.bs * (pr.n_keyframes - pr.n_fixed);
    b.fx = pr.fx; b.fy = pr.fy; b.cx = pr.cx; b.cy = pr.cy;
    char* p = static_cast<char*>(ws);
    b.rec = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.E * b.P * kRec, 256);
    b.SB = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.n * b.n, 256);
    b.SS = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)b.n * b.n, 256);
    b.rhs = reinterpret_cast<float*>(p); p += align_up(sizeof(float) * (size_t)(b.n + 1), 256);
    b.dxi = reinterpret_cast<float*>(p);
    b.cost = cost;
    b.status = pr.status;
    // zero the accumulators (SB, SS, rhs are contiguous after the records)
    const size_t zero_bytes = 2 * align_up(sizeof(float) * (size_t)b.n * b.n, 256) +
                              align_up(sizeof(float) * (size_t)(b.n + 1), 256);
    cudaError_t e = cudaMemsetAsync(b.SB, 0, zero_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cost, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (b.imu != nullptr && b.K > 1)
        k_ba_inertial<<<(unsigned)(b.K - 1), kInerThreads, 0, s>>>(b);
    if (b.E > 0 || b.imu != nullptr) {
        if (b.E > 0)
        k_ba_terms<<<dim3((unsigned)ceil_div(b.P, kTermThreads * kTermPix), (unsigned)b.E), kTermThreads, 0, s>>>(b);
        if (b.n > 0) {
            if (b.E > 0)
                k_ba_schur<<<dim3((unsigned)ceil_div(b.P, kSchurChunk), (unsigned)b.K), kSchurThreads, 0, s>>>(
                    b, lambda, eps);
            const int n_pad = (int)ceil_div(b.n, kNb) * kNb;
            const int cl_rows = cl_panels(n_pad / kNb, 0) * kNb;
            const size_t smem = sizeof(float) * (size_t)(cl_rows + 2 * kNb) * (n_pad + 1);
            const int cpl = (int)ceil_div((int64_t)n_pad + 1 - kNb, 32);
            switch (cpl) {
#define GS_SOLVE(C)                                                                                      \
    case C:                                                                                              \
        e = cudaFuncSetAttribute(k_ba_solve_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 (int)smem);                                                             \
        if (e != cudaSuccess) return e;                                                                  \
        k_ba_solve_cluster<C><<<kClusterCtas, kClSolveThreads, smem, s>>>(b, lambda, eps);               \
        break;
                GS_SOLVE(1)
                GS_SOLVE(2)
                GS_SOLVE(3)
                GS_SOLVE(4)
                GS_SOLVE(5)
                GS_SOLVE(6)
                GS_SOLVE(7)
#undef GS_SOLVE
                default: return cudaErrorInvalidValue;
            }
        }
        k_ba_update<<<dim3((unsigned)ceil_div(b.P, kUpdateThreads), (unsigned)b.K), kUpdateThreads, 0, s>>>(b, lambda,
                                                                                                      eps);
    }
    return cudaGetLastError();
}

}  // namespace gs
