// Row a3 (final stage) and a4: sum the partial moments (the 2D sweep's
// per-warp-task partials, the 1D sweep's per-warp partials) in a fixed order in FP64
// and form the gray low-order closures of Sec. 2
// (Eqs. sigmaE, sigmaF, sigma_P, additive_mg_correction) from them and the
// nodal spectra left by the emission pass.  Also the pack / unpack kernels
// between the canonical intensity I[d][g][cell][node] and the sweep layout
// [quadrant][warp task][cell][slot][lane][node].
#include <algorithm>

#include "sm_internal.cuh"

namespace smk {

// qmom: per-quadrant phi, F_x, F_y and the second moments Pi = sum w Omega
// Omega I (Pi_xx, Pi_xy, Pi_yy) per node, for the consistent method's
// half-range closures; set s belongs to quadrant s / sets_per_q (2D: the sets
// are the quadrants; 1D: the per-warp partials, NWT warps per half, with the
// halves mu > 0 and mu < 0 as quadrants 0 and 1 and phi, F, 0, Pi_xx, 0, 0).
template <typename RT>
__global__ void reduce_kernel(int dim, int nnodes_total, int nm, int nsets, size_t set_stride,
                              double inv_c, const RT *__restrict__ part,
                              const double *__restrict__ gray, double *__restrict__ mom,
                              double *__restrict__ clo, double *__restrict__ qmom,
                              int sets_per_q, const int *__restrict__ active) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // (cell, node)
    if (t >= nnodes_total || (active && *active == 0)) return;
    double acc[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) acc[m] = 0.0;
    double qa[4][6];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 6; ++k) qa[q][k] = 0.0;
    const RT *pp = part + (size_t)t * nm;
    for (int s = 0; s < nsets; ++s) {
        const RT *ps = pp + (size_t)s * set_stride;
        for (int m = 0; m < nm; ++m) acc[m] += (double)ps[m];
        if (qmom) {
            const int q = min(s / sets_per_q, 3);
            if (dim == 2) {
                for (int k = 0; k < 6; ++k) qa[q][k] += (double)ps[k];
            } else {
                qa[q][0] += (double)ps[0];
                qa[q][1] += (double)ps[1];
                qa[q][3] += (double)ps[2];
            }
        }
    }
    if (qmom) {
        for (int q = 0; q < 4; ++q) {
            double *o = qmom + ((size_t)t * 4 + q) * 6;
            const double ph = qa[q][0];
            o[0] = ph;
            o[1] = qa[q][1];
            o[2] = qa[q][2];
            o[3] = qa[q][3] + ph / 3.0;
            o[4] = qa[q][4];
            o[5] = dim == 2 ? qa[q][5] + ph / 3.0 : 0.0;
        }
    }
    if (mom) {
        for (int m = 0; m < nm; ++m) mom[(size_t)t * nm + m] = acc[m];
    }
    if (clo) {
        const double sP = gray[(size_t)t * 2 + 0], sF = gray[(size_t)t * 2 + 1];
        const double phi = acc[0];
        if (dim == 1) {
            double *o = clo + (size_t)t * 7;
            o[0] = phi * inv_c;
            o[1] = acc[1];
            o[2] = acc[2];
            o[3] = (phi > 0.0 && acc[3] > 0.0) ? acc[3] / phi : sP;
            o[4] = sF;
            o[5] = sP;
            o[6] = sF * acc[1] - acc[4];
        } else {
            double *o = clo + (size_t)t * 11;
            o[0] = phi * inv_c;
            o[1] = acc[1];
            o[2] = acc[2];
            o[3] = acc[3];
            o[4] = acc[4];
            o[5] = acc[5];
            o[6] = (phi > 0.0 && acc[6] > 0.0) ? acc[6] / phi : sP;
            o[7] = sF;
            o[8] = sP;
            o[9] = sF * acc[1] - acc[7];
            o[10] = sF * acc[2] - acc[8];
        }
    }
}

// The 2D form: the partials are [set][cell][36] (36 = 4 nodes x 9 moments, one
// set per warp task).  A block of 8 cells x 36 slots: thread (cell, slot) sums
// its slot over the sets in order (coalesced: the block reads 288 consecutive
// values per set), the per-quadrant sums too when qmom is wanted; then one
// thread per node forms the node's moments and closures from shared memory.
constexpr int RCELLS = 8;

// A fixed-order sum of the sets.  FP32 partials are summed as an unevaluated
// pair (s, c) of FP32 numbers: TwoSum (Knuth) yields each addition's rounding
// error exactly and the errors are summed on the side (Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005: Sum2), so the pair carries the sum to
// about twice FP32's precision at FP32 cost and becomes one FP64 value once per
// slot.  On this GPU an FP64 add or conversion issues at 1/64 of the FP32 rate:
// an FP64 running sum (a conversion and an add per set) made the reduction
// FP64-bound at a sixth of the HBM bandwidth.
template <typename RT> struct SetSum;
template <> struct SetSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct SetSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x);
        const float z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename RT>
__global__ void __launch_bounds__(RCELLS * 36)
reduce2d_kernel(int ncell, int nsets, double inv_c, const RT *__restrict__ part,
                const double *__restrict__ gray, double *__restrict__ mom,
                double *__restrict__ clo, double *__restrict__ qmom, int sets_per_q,
                const int *__restrict__ active) {
    if (active && *active == 0) return;  // a batch member that is not swept this pass
    __shared__ double s_sum[RCELLS][36];
    __shared__ double s_q[RCELLS][4][24];  // per quadrant: nodes x {phi, Fx, Fy, Pxx, Pxy, Pyy}
    const int c = threadIdx.x / 36, m = threadIdx.x - 36 * c;
    const int cell = blockIdx.x * RCELLS + c;
    const size_t stride = (size_t)ncell * 36;
    double acc = 0.0;
    if (cell < ncell) {
        const RT *pp = part + (size_t)cell * 36 + m;
        const int k = m % 9;
        if (qmom && k < 6) {
            for (int q = 0; q < 4; ++q) {
                SetSum<RT> qa;
                const int s0 = min(q * sets_per_q, nsets), s1 = q == 3 ? nsets : min(s0 + sets_per_q, nsets);
                for (int s = s0; s < s1; ++s) qa.add(pp[(size_t)s * stride]);
                s_q[c][q][(m / 9) * 6 + k] = qa.value();
                acc += qa.value();
            }
        } else {
            SetSum<RT> sum;
            int s = 0;
            for (; s + 4 <= nsets; s += 4) {
                const RT a0 = pp[(size_t)s * stride];
                const RT a1 = pp[(size_t)(s + 1) * stride];
                const RT a2 = pp[(size_t)(s + 2) * stride];
                const RT a3 = pp[(size_t)(s + 3) * stride];
                sum.add(a0);
                sum.add(a1);
                sum.add(a2);
                sum.add(a3);
            }
            for (; s < nsets; ++s) sum.add(pp[(size_t)s * stride]);
            acc = sum.value();
        }
    }
    s_sum[c][m] = acc;
    __syncthreads();
    if (threadIdx.x >= RCELLS * 4) return;
    const int cc = threadIdx.x >> 2, node = threadIdx.x & 3;
    const int cl = blockIdx.x * RCELLS + cc;
    if (cl >= ncell) return;
    const size_t t = (size_t)cl * 4 + node;
    const double *a = &s_sum[cc][node * 9];
    if (qmom) {
        for (int q = 0; q < 4; ++q) {
            const double *v = &s_q[cc][q][node * 6];
            double *o = qmom + (t * 4 + q) * 6;
            const double ph = v[0];
            o[0] = ph;
            o[1] = v[1];
            o[2] = v[2];
            o[3] = v[3] + ph / 3.0;
            o[4] = v[4];
            o[5] = v[5] + ph / 3.0;
        }
    }
    if (mom)
        for (int k = 0; k < 9; ++k) mom[t * 9 + k] = a[k];
    if (clo) {
        const double sP = gray[t * 2 + 0], sF = gray[t * 2 + 1];
        const double phi = a[0];
        double *o = clo + t * 11;
        o[0] = phi * inv_c;
        o[1] = a[1];
        o[2] = a[2];
        o[3] = a[3];
        o[4] = a[4];
        o[5] = a[5];
        o[6] = (phi > 0.0 && a[6] > 0.0) ? a[6] / phi : sP;
        o[7] = sF;
        o[8] = sP;
        o[9] = sF * a[1] - a[7];
        o[10] = sF * a[2] - a[8];
    }
}

// The 2D reduction of partials in precision prec (the FP32 correction sweeps
// of an FP64 problem's defect correction).
cudaError_t launch_reduce_prec(int prec, const sm_problem *p, const void *part, int n_part,
                               double *mom, double *clo, cudaStream_t s) {
    const int blocks = (p->ncell + RCELLS - 1) / RCELLS;
    const double inv_c = 1.0 / p->desc.c;
    if (prec == 32)
        reduce2d_kernel<float><<<blocks, RCELLS * 36, 0, s>>>(
            p->ncell, n_part, inv_c, (const float *)part, p->d_gray, mom, clo, nullptr, 1, nullptr);
    else
        reduce2d_kernel<double><<<blocks, RCELLS * 36, 0, s>>>(
            p->ncell, n_part, inv_c, (const double *)part, p->d_gray, mom, clo, nullptr, 1,
            nullptr);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const sm_problem *p, const void *part, int n_part, double *mom,
                          double *clo, cudaStream_t s, double *qmom, int sets_per_q,
                          const int *active) {
    const int n = p->ncell * p->nn;
    const int threads = 128;
    const size_t stride = (size_t)n * p->nm;
    const double inv_c = 1.0 / p->desc.c;
    if (p->dim == 2) {
        const int blocks = (p->ncell + RCELLS - 1) / RCELLS;
        if (p->prec == 32)
            reduce2d_kernel<float><<<blocks, RCELLS * 36, 0, s>>>(
                p->ncell, n_part, inv_c, (const float *)part, p->d_gray, mom, clo, qmom, sets_per_q,
                active);
        else
            reduce2d_kernel<double><<<blocks, RCELLS * 36, 0, s>>>(
                p->ncell, n_part, inv_c, (const double *)part, p->d_gray, mom, clo, qmom,
                sets_per_q, active);
        return cudaGetLastError();
    }
    if (p->prec == 32)
        reduce_kernel<float><<<(n + threads - 1) / threads, threads, 0, s>>>(
            p->dim, n, p->nm, n_part, stride, inv_c, (const float *)part, p->d_gray, mom, clo,
            qmom, sets_per_q, active);
    else
        reduce_kernel<double><<<(n + threads - 1) / threads, threads, 0, s>>>(
            p->dim, n, p->nm, n_part, stride, inv_c, (const double *)part, p->d_gray, mom, clo,
            qmom, sets_per_q, active);
    return cudaGetLastError();
}

template <typename RT>
__global__ void pack_kernel(size_t total, int nn, int ncell, int GW, int NWT, int NGB, int LG,
                            int DB, int G, const int *__restrict__ dir_of,
                            const LaneConst *__restrict__ lanes, double *__restrict__ canon,
                            RT *__restrict__ packed, int unpack) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        size_t e = idx;
        const int node = (int)(e % nn);
        e /= nn;
        const int lane = (int)(e % 32);
        e /= 32;
        const int gw = (int)(e % GW);
        e /= GW;
        const int cell = (int)(e % ncell);
        e /= ncell;
        const int wt = (int)(e % NWT);
        const int q = (int)(e / NWT);
        const int db = wt / NGB, gb = wt - db * NGB;
        const int li = (q * DB + db) * 32 + lane;
        const int d = dir_of[li];
        const int g = gb * GW * LG + gw * LG + lanes[li].g_lo;
        const bool valid = d >= 0 && g < G;
        const size_t ci = (((size_t)d * G + g) * ncell + cell) * nn + node;
        if (!unpack) {
            packed[idx] = valid ? (RT)canon[ci] : (RT)0;
        } else if (valid) {
            canon[ci] = (double)packed[idx];
        }
    }
}

cudaError_t launch_pack(const sm_problem *p, const double *canon, void *packed, int unpack,
                        cudaStream_t s) {
    const size_t total = (size_t)p->NQ * p->NWT * p->ncell * p->GW * 32 * p->nn;
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((total + threads - 1) / threads, 65535 * 8);
    if (p->prec == 32)
        pack_kernel<float><<<blocks, threads, 0, s>>>(total, p->nn, p->ncell, p->GW, p->NWT, p->NGB,
                                                      p->LG, p->DB, p->G, p->d_dir_of, p->d_lanes,
                                                      const_cast<double *>(canon), (float *)packed,
                                                      unpack);
    else
        pack_kernel<double><<<blocks, threads, 0, s>>>(total, p->nn, p->ncell, p->GW, p->NWT,
                                                       p->NGB, p->LG, p->DB, p->G, p->d_dir_of,
                                                       p->d_lanes, const_cast<double *>(canon),
                                                       (double *)packed, unpack);
    return cudaGetLastError();
}

}  // namespace smk
