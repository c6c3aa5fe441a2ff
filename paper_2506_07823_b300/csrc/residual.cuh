// residual.cuh -- FP64 residual of the LQ KKT system and the update of one
// iterative-refinement step.
//
// For z = (dx, du, dlam) the KKT rows (first-order conditions of Eq. (QP)
// with the Lagrangian of Sec. II-B) are
//   init      s - dx_0                                        = 0
//   x_k       Q dx_k + S^T du_k + q_k + A^T dlam_{k+1} - dlam_k = 0   (k < N)
//   u_k       S dx_k + R du_k + r_k + B^T dlam_{k+1}          = 0   (k < N)
//   dyn_k     A dx_k + B du_k + c_k - dx_{k+1}                = 0   (k < N)
//   term      Q_N dx_N + q_N - dlam_N                         = 0
// Every row is evaluated in double precision from the FP32 data.  The rows
// are also the right-hand side of the correction system: K dz = -rows means
// an LQ problem with the same matrices and vectors
//   s' = s - dx_0, q' = row_x (row_term at N), r' = row_u, c' = row_dyn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kkt_scan.cuh"

namespace pdl {

struct ResidArgs {
    const float *A, *B, *c, *Q, *R, *S, *q, *r, *s;
    const float *dx, *du, *dlam;
    const int32_t* N;
    const int64_t* off;
    const int64_t* stage_inst;   // [total stages] owning instance of each slot, -1 if none
    int64_t total_stages;
    double* norms;               // [count][4]: |res|, |K|, |z|, |rhs| (max-reduced)
    float *rq, *rr, *rc, *rs;    // optional correction right-hand side (null: skip)
};

__device__ __forceinline__ void atomic_max_pos(double* addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per stage slot; lanes own rows.
template <int NX, int NU>
__global__ void __launch_bounds__(256) kkt_residual_kernel(const __grid_constant__ ResidArgs a)
{
    const int64_t gs = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (gs >= a.total_stages) return;
    const int64_t inst = a.stage_inst[gs];
    if (inst < 0) return;  // slot between instances
    const int N = a.N[inst];
    const int k = (int)(gs - a.off[inst]);
    double res = 0.0, kn = 0.0, zn = 0.0, rn = 0.0;
    const float* dx = a.dx + gs * NX;
    const float* dl = a.dlam + gs * NX;
    if (k < N) {
        const float* A = a.A + gs * NX * NX;
        const float* B = a.B + gs * NX * NU;
        const float* Q = a.Q + gs * NX * NX;
        const float* R = a.R + gs * NU * NU;
        const float* S = a.S ? a.S + gs * NU * NX : nullptr;
        const float* du = a.du + gs * NU;
        const float* dx1 = a.dx + (gs + 1) * NX;
        const float* dl1 = a.dlam + (gs + 1) * NX;
        for (int i = lane; i < NX; i += 32) {
            // x-row
            double v = (double)a.q[gs * NX + i] - (double)dl[i], row = 1.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)Q[i * NX + j] * (double)dx[j] + (double)A[j * NX + i] * (double)dl1[j];
                row += fabs((double)Q[i * NX + j]) + fabs((double)A[j * NX + i]);
            }
            if (S)
                for (int j = 0; j < NU; ++j) {
                    v += (double)S[j * NX + i] * (double)du[j];
                    row += fabs((double)S[j * NX + i]);
                }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.q[gs * NX + i]));
            if (a.rq) a.rq[gs * NX + i] = (float)v;
            // dynamics row
            double d = (double)a.c[gs * NX + i] - (double)dx1[i];
            row = 1.0;
            for (int j = 0; j < NX; ++j) {
                d += (double)A[i * NX + j] * (double)dx[j];
                row += fabs((double)A[i * NX + j]);
            }
            for (int j = 0; j < NU; ++j) {
                d += (double)B[i * NU + j] * (double)du[j];
                row += fabs((double)B[i * NU + j]);
            }
            res = fmax(res, fabs(d));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.c[gs * NX + i]));
            if (a.rc) a.rc[gs * NX + i] = (float)d;
            zn = fmax(zn, fmax(fabs((double)dx[i]), fabs((double)dl[i])));
        }
        for (int i = lane; i < NU; i += 32) {
            double v = (double)a.r[gs * NU + i], row = 0.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)B[j * NU + i] * (double)dl1[j];
                row += fabs((double)B[j * NU + i]);
                if (S) {
                    v += (double)S[i * NX + j] * (double)dx[j];
                    row += fabs((double)S[i * NX + j]);
                }
            }
            for (int j = 0; j < NU; ++j) {
                v += (double)R[i * NU + j] * (double)du[j];
                row += fabs((double)R[i * NU + j]);
            }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.r[gs * NU + i]));
            if (a.rr) a.rr[gs * NU + i] = (float)v;
            zn = fmax(zn, fabs((double)du[i]));
        }
    } else {
        const float* Q = a.Q + gs * NX * NX;
        for (int i = lane; i < NX; i += 32) {
            double v = (double)a.q[gs * NX + i] - (double)dl[i], row = 1.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)Q[i * NX + j] * (double)dx[j];
                row += fabs((double)Q[i * NX + j]);
            }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.q[gs * NX + i]));
            if (a.rq) a.rq[gs * NX + i] = (float)v;
            zn = fmax(zn, fmax(fabs((double)dx[i]), fabs((double)dl[i])));
        }
        if (a.rr)
            for (int i = lane; i < NU; i += 32) a.rr[gs * NU + i] = 0.f;
        if (a.rc)
            for (int i = lane; i < NX; i += 32) a.rc[gs * NX + i] = 0.f;
    }
    if (k == 0) {
        for (int i = lane; i < NX; i += 32) {
            const double sv = (double)a.s[inst * NX + i];
            const double d = sv - (double)dx[i];
            res = fmax(res, fabs(d));
            kn = fmax(kn, 1.0);
            rn = fmax(rn, fabs(sv));
            if (a.rs) a.rs[inst * NX + i] = (float)d;
        }
    }
    res = warp_max(res);
    kn = warp_max(kn);
    zn = warp_max(zn);
    rn = warp_max(rn);
    if (lane == 0) {
        double* o = a.norms + inst * 4;
        atomic_max_pos(o + 0, res);
        atomic_max_pos(o + 1, kn);
        atomic_max_pos(o + 2, zn);
        atomic_max_pos(o + 3, rn);
    }
}

// ---------------------------------------------------------------------------
// The same rows with the stage matrices staged in shared memory, for sizes
// whose SPB stages fit: the block copies SPB consecutive stage slots with
// coalesced 16-byte loads into row-padded areas (odd row strides, so that
// both row and column walks are free of bank conflicts) and the vectors as
// doubles, then one thread per KKT row evaluates it.  The threads are split
// into three warp-aligned segments -- x-rows, dynamics rows, u-rows of all
// SPB stages -- so that no warp mixes row kinds.  Products of two FP32 values
// are exact in FP64 and accumulate by DFMA; the absolute row sums (the
// matrix norm of the backward error) accumulate in compensated FP32 (TwoSum,
// about 2^-48 relative), off the FP64 pipe.
template <int NX, int NU>
struct ResStage {
    static constexpr int LQ = NX + 1, LU = NU + 1;     // padded row strides
    static constexpr int Q = 0, A = Q + NX * LQ, B = A + NX * LQ, R = B + NX * LU,
                         S = R + NU * LU, FLOATS = round4(S + NU * LQ);
    // doubles after the floats: dx, dx1, dl, dl1 (NX each), du (NU)
    static constexpr int DX = 0, DX1 = NX, DL = 2 * NX, DL1 = 3 * NX, DU = 4 * NX,
                         DOUBLES = 4 * NX + NU + (4 * NX + NU) % 2;
    static constexpr size_t BYTES = sizeof(float) * FLOATS + sizeof(double) * DOUBLES;
};

template <int NX, int NU>
struct ResSmemCfg {
    static constexpr int SPB = 4;                                  // stage slots per block
    static constexpr int XT = (SPB * NX + 31) / 32 * 32, DT = XT, UT = (SPB * NU + 31) / 32 * 32;
    static constexpr int THREADS = XT + DT + UT;
    static constexpr size_t STAGE_BYTES = (ResStage<NX, NU>::BYTES + 15) / 16 * 16;
    static constexpr size_t BYTES = SPB * STAGE_BYTES + SPB * 4 * sizeof(double);
    static constexpr bool value = NX <= 48 && THREADS <= 1024 && BYTES <= 110 * 1024;
};

// Exact binary32 -> binary64 conversion on the integer pipe (IEEE 754 formats:
// sign kept, exponent rebiased from 127 to 1023, the 23 fraction bits become
// the top of the 52).  Zero and subnormal inputs give a signed zero (a
// subnormal FP32 entry, below 1.2e-38, contributes nothing at FP64 scale of
// the residual), infinities and NaNs stay infinities and NaNs.  The FP64
// pipe is left to the DFMAs of the residual rows.
__device__ __forceinline__ double f32_to_f64_int(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t sign = b & 0x80000000u;
    const uint32_t exp64 = e == 0xffu ? 0x7ffu : e + 896u;
    const uint32_t hi = e == 0u ? sign : (sign | (exp64 << 20) | ((b >> 3) & 0xfffffu));
    const uint32_t lo = e == 0u ? 0u : (b << 29);
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

template <int NX, int NU>
__global__ void __launch_bounds__(ResSmemCfg<NX, NU>::THREADS)
kkt_residual_smem_kernel(const __grid_constant__ ResidArgs a)
{
    using C = ResSmemCfg<NX, NU>;
    using L = ResStage<NX, NU>;
    constexpr int SPB = C::SPB;
    extern __shared__ __align__(16) unsigned char rsm[];
    const int t = threadIdx.x;
    const int64_t gs0 = (int64_t)blockIdx.x * SPB;
    const bool hasS = a.S != nullptr;
    double* red = reinterpret_cast<double*>(rsm + SPB * C::STAGE_BYTES);   // [SPB][4]
    for (int e = t; e < SPB * 4; e += C::THREADS) red[e] = 0.0;
    // ---- stage the matrices and vectors of the SPB slots
    for (int s = 0; s < SPB; ++s) {
        const int64_t gs = gs0 + s;
        if (gs >= a.total_stages) break;
        const int64_t inst = a.stage_inst[gs];
        if (inst < 0) continue;
        const bool term = gs - a.off[inst] == a.N[inst];
        float* f = reinterpret_cast<float*>(rsm + s * C::STAGE_BYTES);
        double* d = reinterpret_cast<double*>(f + L::FLOATS);
        auto stage = [&](float* dst, const float* src, int rows, int cols, int ld) {
            for (int e = t; e < rows * cols / 4; e += C::THREADS) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(src) + e);
                const int r = (4 * e) / cols, c = (4 * e) % cols;   // cols % 4 == 0
                float* o = dst + r * ld + c;
                o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
            }
        };
        stage(f + L::Q, a.Q + gs * NX * NX, NX, NX, L::LQ);
        if (!term) {
            stage(f + L::A, a.A + gs * NX * NX, NX, NX, L::LQ);
            stage(f + L::B, a.B + gs * NX * NU, NX, NU, L::LU);
            stage(f + L::R, a.R + gs * NU * NU, NU, NU, L::LU);
            if (hasS) stage(f + L::S, a.S + gs * NU * NX, NU, NX, L::LQ);
        }
        for (int i = t; i < NX; i += C::THREADS) {
            d[L::DX + i] = (double)a.dx[gs * NX + i];
            d[L::DL + i] = (double)a.dlam[gs * NX + i];
            if (!term) {
                d[L::DX1 + i] = (double)a.dx[(gs + 1) * NX + i];
                d[L::DL1 + i] = (double)a.dlam[(gs + 1) * NX + i];
            }
        }
        if (!term)
            for (int i = t; i < NU; i += C::THREADS) d[L::DU + i] = (double)a.du[gs * NU + i];
    }
    __syncthreads();
    // ---- one thread per row
    int seg, rho;
    if (t < C::XT) { seg = 0; rho = t; }
    else if (t < C::XT + C::DT) { seg = 1; rho = t - C::XT; }
    else { seg = 2; rho = t - C::XT - C::DT; }
    const int per = seg == 2 ? NU : NX;
    const int s = rho / per, i = rho % per;
    const int64_t gs = gs0 + s;
    int64_t inst = -1;
    if (s < SPB && gs < a.total_stages) inst = a.stage_inst[gs];
    if (inst >= 0) {
        const int k = (int)(gs - a.off[inst]);
        const bool term = k == a.N[inst];
        const float* f = reinterpret_cast<const float*>(rsm + s * C::STAGE_BYTES);
        const double* d = reinterpret_cast<const double*>(f + L::FLOATS);
        double res = 0.0, kn = 0.0, zn = 0.0, rn = 0.0;
        float hi = 0.f, lo = 0.f;
        if (seg == 0) {
            // x-row i (terminal: Q_N dx_N + q_N - dlam_N)
            const double qi = (double)a.q[gs * NX + i];
            double v = qi - d[L::DL + i];
            hi = 1.f;
            for (int j = 0; j < NX; ++j) {
                const float qij = f[L::Q + i * L::LQ + j];
                v = fma(f32_to_f64_int(qij), d[L::DX + j], v);
                two_sum_acc(hi, lo, fabsf(qij));
            }
            if (!term) {
                for (int j = 0; j < NX; ++j) {
                    const float aji = f[L::A + j * L::LQ + i];
                    v = fma(f32_to_f64_int(aji), d[L::DL1 + j], v);
                    two_sum_acc(hi, lo, fabsf(aji));
                }
                if (hasS)
                    for (int j = 0; j < NU; ++j) {
                        const float sji = f[L::S + j * L::LQ + i];
                        v = fma(f32_to_f64_int(sji), d[L::DU + j], v);
                        two_sum_acc(hi, lo, fabsf(sji));
                    }
            }
            res = fabs(v);
            rn = fabs(qi);
            zn = fmax(fabs(d[L::DX + i]), fabs(d[L::DL + i]));
            if (a.rq) a.rq[gs * NX + i] = (float)v;
            if (k == 0) {
                const double sv = (double)a.s[inst * NX + i];
                const double dd = sv - d[L::DX + i];
                res = fmax(res, fabs(dd));
                kn = 1.0;
                rn = fmax(rn, fabs(sv));
                if (a.rs) a.rs[inst * NX + i] = (float)dd;
            }
        } else if (seg == 1) {
            // dynamics row i: A dx + B du + c - dx_{k+1}
            if (!term) {
                const double ci = (double)a.c[gs * NX + i];
                double v = ci - d[L::DX1 + i];
                hi = 1.f;
                for (int j = 0; j < NX; ++j) {
                    const float aij = f[L::A + i * L::LQ + j];
                    v = fma(f32_to_f64_int(aij), d[L::DX + j], v);
                    two_sum_acc(hi, lo, fabsf(aij));
                }
                for (int j = 0; j < NU; ++j) {
                    const float bij = f[L::B + i * L::LU + j];
                    v = fma(f32_to_f64_int(bij), d[L::DU + j], v);
                    two_sum_acc(hi, lo, fabsf(bij));
                }
                res = fabs(v);
                rn = fabs(ci);
                if (a.rc) a.rc[gs * NX + i] = (float)v;
            } else if (a.rc) {
                a.rc[gs * NX + i] = 0.f;
            }
        } else {
            // u-row i: S dx + R du + r + B^T dlam_{k+1}
            if (!term) {
                const double ri = (double)a.r[gs * NU + i];
                double v = ri;
                for (int j = 0; j < NX; ++j) {
                    const float bji = f[L::B + j * L::LU + i];
                    v = fma(f32_to_f64_int(bji), d[L::DL1 + j], v);
                    two_sum_acc(hi, lo, fabsf(bji));
                }
                if (hasS)
                    for (int j = 0; j < NX; ++j) {
                        const float sij = f[L::S + i * L::LQ + j];
                        v = fma(f32_to_f64_int(sij), d[L::DX + j], v);
                        two_sum_acc(hi, lo, fabsf(sij));
                    }
                for (int j = 0; j < NU; ++j) {
                    const float rij = f[L::R + i * L::LU + j];
                    v = fma(f32_to_f64_int(rij), d[L::DU + j], v);
                    two_sum_acc(hi, lo, fabsf(rij));
                }
                res = fabs(v);
                rn = fabs(ri);
                zn = fabs(d[L::DU + i]);
                if (a.rr) a.rr[gs * NU + i] = (float)v;
            } else if (a.rr) {
                a.rr[gs * NU + i] = 0.f;
            }
        }
        kn = fmax(kn, (double)hi + (double)lo);
        double* o = red + s * 4;
        atomic_max_pos(o + 0, res);
        atomic_max_pos(o + 1, kn);
        atomic_max_pos(o + 2, zn);
        atomic_max_pos(o + 3, rn);
    }
    __syncthreads();
    if (t < SPB * 4) {
        const int s2 = t / 4, c = t % 4;
        const int64_t g2 = gs0 + s2;
        if (g2 < a.total_stages) {
            const int64_t in2 = a.stage_inst[g2];
            if (in2 >= 0) atomic_max_pos(a.norms + in2 * 4 + c, red[s2 * 4 + c]);
        }
    }
}

// z += dz over n elements (one refinement update).
static __global__ void axpy_kernel(float* __restrict__ z, const float* __restrict__ dz, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] += dz[i];
}

}  // namespace pdl
