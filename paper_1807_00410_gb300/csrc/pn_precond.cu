// Learned preconditioner glue: P_N vectors <-> network tensors, and the
// preconditioner application used inside flexible GMRES.
//
//   M(v) = s net(features(v / s)) + P v,   s = |v| / sqrt(n) (RMS of v over
//   the n unknowns, so the network sees values of order one)
//
// P is a fixed row-scaled diagonal, P = diag(1 / (D + 1/h)) with D the
// collision-minus-scattering diagonal and 1/h the scale of the transport
// couplings of a row: in optically thick cells it is the Jacobi inverse
// D^{-1}, in thin cells (where D^{-1} would amplify every rough component by
// 1/D) it is h times the identity.  P covers every unknown, including the
// x = R, y = R, z = R face slots the network does not see, so M is never
// rank-deficient.
//
// features(u) at voxel (x, y, z) < R: channel p = u of plane p at slot
// (x, y, z) (the cell's own slot on every staggered grid), then
// log(sigma_t h), sigma_s / sigma_t and g.  The network's K output channels
// go back to slot (x, y, z) of each plane.  Training either fits pairs
// (r, e) with A e = r (target (e - P r) / s) or minimises |A M(r) - r|^2 /
// |r|^2 directly, with the gradient A^T (A M(r) - r) gathered back to the
// cell slots (pn_cnn_output, pn_cnn_targets).
#include <cuda_runtime.h>

#include <cmath>

#include "pn_internal.h"

extern "C" int pn_cnn_forward(struct pn_cnn* net, const float* in, float* out, int B, int Z, int Y, int X,
                              void* stream);

namespace {

__device__ __forceinline__ float centre_mean_f(const float* F, int R, int x, int y, int z, int px, int py, int pz) {
    const int x0 = px ? max(x - 1, 0) : x, x1 = px ? min(x, R - 1) : x;
    const int y0 = py ? max(y - 1, 0) : y, y1 = py ? min(y, R - 1) : y;
    const int z0 = pz ? max(z - 1, 0) : z, z1 = pz ? min(z, R - 1) : z;
    const int64_t R2 = int64_t(R) * R;
    return 0.125f * (F[z0 * R2 + y0 * R + x0] + F[z0 * R2 + y0 * R + x1] + F[z0 * R2 + y1 * R + x0] +
                     F[z0 * R2 + y1 * R + x1] + F[z1 * R2 + y0 * R + x0] + F[z1 * R2 + y0 * R + x1] +
                     F[z1 * R2 + y1 * R + x0] + F[z1 * R2 + y1 * R + x1]);
}

// D + 1/h at slot (x, y, z) of plane P (the fixed part's row scale)
__device__ __forceinline__ float fixed_row(const float* st, const float* ss, int R, int x, int y, int z,
                                           const pn::Plane& P) {
    return centre_mean_f(st, R, x, y, z, P.px, P.py, P.pz) - P.fl_f * centre_mean_f(ss, R, x, y, z, P.px, P.py, P.pz) +
           float(R);
}

struct FeatArgs {
    const float* u;       // padded vector
    const double* nrm2;   // device |u|^2 (scale = sqrt(n_unknowns)/|u|) or null
    double scale;         // used when nrm2 is null
    const float* st;
    const float* ss;
    float g;
    int R, K;
    int64_t pitch_x, pitch_y, plane_stride;
    float* out;           // [R^3][K + 3]
};

__global__ void k_features(FeatArgs a) {
    const int C = a.K + 3;
    const int64_t V = int64_t(a.R) * a.R * a.R;
    float sc = float(a.scale);
    if (a.nrm2) {
        const double n2 = *a.nrm2;
        sc = n2 > 0.0 ? float(a.scale / sqrt(n2)) : 0.0f;
    }
    const float h = 1.0f / a.R;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < V * C; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % C);
        const int64_t v = i / C;
        const int x = int(v % a.R), y = int((v / a.R) % a.R), z = int(v / (int64_t(a.R) * a.R));
        float val;
        if (c < a.K) {
            val = sc * a.u[int64_t(c) * a.plane_stride + z * a.pitch_y + y * a.pitch_x + x];
        } else if (c == a.K) {
            val = logf(fmaxf(a.st[v] * h, 1e-12f));
        } else if (c == a.K + 1) {
            val = a.st[v] > 0.0f ? a.ss[v] / a.st[v] : 0.0f;
        } else {
            val = a.g;
        }
        a.out[i] = val;
    }
}

// z = scale * net_out (slots < R) + P v over the whole padded vector (either
// term may be absent).
struct ScatterArgs {
    const float* net_out;  // [R^3][K] or null
    const double* nrm2;    // device |v|^2: scale = |v| * scale field (or null: scale field)
    double scale;
    const float* v;        // vector for the Jacobi term (or null)
    float* z;              // padded output
    const pn::Plane* planes;
    const float* st;
    const float* ss;
    int R, K;
    int64_t pitch_x, pitch_y, plane_stride;
};

__global__ void k_scatter(ScatterArgs a) {
    const int64_t n = a.plane_stride * a.K;
    const int R = a.R;
    float sc = float(a.scale);
    if (a.nrm2) sc = float(a.scale * sqrt(fmax(*a.nrm2, 0.0)));
    const int64_t box = a.pitch_y * (R + 1);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int p = int(i / a.plane_stride);
        const int64_t s = i % a.plane_stride;
        float out = 0.0f;
        if (s < box) {
            const int x = int(s % a.pitch_x);
            const int64_t t = s / a.pitch_x;
            const int y = int(t % (R + 1)), zz = int(t / (R + 1));
            const pn::Plane P = a.planes[p];
            if (x < R + P.px && y < R + P.py && zz < R + P.pz) {
                if (a.net_out && x < R && y < R && zz < R)
                    out = sc * a.net_out[((int64_t(zz) * R + y) * R + x) * a.K + p];
                if (a.v) out += a.v[i] / fixed_row(a.st, a.ss, R, x, y, zz, P);
            }
        }
        a.z[i] = out;
    }
}

// target[v][c] = scale * (e - P r) at the cell's own slots (r may be null:
// scale * e, the gather of a padded vector to the network's layout)
__global__ void k_targets(const float* e, const float* r, float scale, const pn::Plane* planes, const float* st,
                          const float* ss, int R, int K, int64_t pitch_x, int64_t pitch_y, int64_t plane_stride,
                          float* out) {
    const int64_t V = int64_t(R) * R * R;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < V * K; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % K);
        const int64_t v = i / K;
        const int x = int(v % R), y = int((v / R) % R), z = int(v / (int64_t(R) * R));
        const pn::Plane P = planes[c];
        const int64_t off = int64_t(c) * plane_stride + z * pitch_y + y * pitch_x + x;
        out[i] = r ? scale * (e[off] - r[off] / fixed_row(st, ss, R, x, y, z, P)) : scale * e[off];
    }
}

int grid_for(int64_t n) { return int(std::min<int64_t>(16 * 1024, std::max<int64_t>(1, (n + 255) / 256))); }

}  // namespace

namespace pn {

// z = M(v) with the network net; scratch holds the features and the network
// output (R^3 (2K + 3) floats); nrm2_dev receives |v|^2.
int precond_apply(pn_handle* h, struct pn_cnn* net, const float* v, float* z, float* scratch, double* nrm2_dev,
                  cudaStream_t s) {
    const int R = h->R, K = h->K;
    const int64_t V = int64_t(R) * R * R;
    cudaError_t e = launch_dot(h, v, v, h->n_elems, PN_F32, nrm2_dev, s);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "precond: norm");
    float* feat = scratch;
    float* out = scratch + V * (K + 3);
    const double rms_n = std::sqrt(double(h->n_active));
    FeatArgs fa{v, nrm2_dev, rms_n, h->d_st_f, h->d_ss_f, float(h->g), R, K, h->pitch_x, h->pitch_y, h->plane_stride,
                feat};
    k_features<<<grid_for(V * (K + 3)), 256, 0, s>>>(fa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "precond: features");
    const int rc = pn_cnn_forward(net, feat, out, 1, R, R, R, s);
    if (rc != PN_OK) return pn_fail(h, rc, "precond: network forward failed");
    ScatterArgs sa{out, nrm2_dev, 1.0 / rms_n, v, z, h->d_planes, h->d_st_f, h->d_ss_f, R, K, h->pitch_x, h->pitch_y,
                   h->plane_stride};
    k_scatter<<<grid_for(h->n_elems), 256, 0, s>>>(sa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "precond: scatter");
    return PN_OK;
}

}  // namespace pn

extern "C" {

int pn_cnn_features(pn_handle* h, const float* v, double scale, float* out, void* stream) {
    if (!h || !v || !out) return PN_ERR_ARG;
    if (h->dims != 3 || h->periodic)
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_cnn_features: 3D vacuum-boundary handles only");
    const int64_t V = int64_t(h->R) * h->R * h->R;
    FeatArgs fa{v, nullptr, scale, h->d_st_f, h->d_ss_f, float(h->g), h->R, h->K, h->pitch_x, h->pitch_y,
                h->plane_stride, out};
    k_features<<<grid_for(V * (h->K + 3)), 256, 0, (cudaStream_t)stream>>>(fa);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PN_OK : pn_cuda_fail(h, e, "pn_cnn_features");
}

int pn_cnn_targets(pn_handle* h, const float* e, const float* r, double scale, float* out, void* stream) {
    if (!h || !e || !out) return PN_ERR_ARG;
    if (h->dims != 3 || h->periodic)
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_cnn_targets: 3D vacuum-boundary handles only");
    const int64_t V = int64_t(h->R) * h->R * h->R;
    k_targets<<<grid_for(V * h->K), 256, 0, (cudaStream_t)stream>>>(e, r, float(scale), h->d_planes, h->d_st_f,
                                                                      h->d_ss_f, h->R, h->K, h->pitch_x, h->pitch_y,
                                                                      h->plane_stride, out);
    const cudaError_t er = cudaGetLastError();
    return er == cudaSuccess ? PN_OK : pn_cuda_fail(h, er, "pn_cnn_targets");
}

int pn_cnn_output(pn_handle* h, const float* net_out, double scale, const float* v, float* z, void* stream) {
    if (!h || !z) return PN_ERR_ARG;
    if (h->dims != 3 || h->periodic)
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_cnn_output: 3D vacuum-boundary handles only");
    ScatterArgs sa{net_out, nullptr, scale, v, z, h->d_planes, h->d_st_f, h->d_ss_f, h->R, h->K, h->pitch_x,
                   h->pitch_y, h->plane_stride};
    k_scatter<<<grid_for(h->n_elems), 256, 0, (cudaStream_t)stream>>>(sa);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PN_OK : pn_cuda_fail(h, e, "pn_cnn_output");
}

int pn_cnn_precondition(pn_handle* h, struct pn_cnn* net, const float* v, float* z, void* stream) {
    if (!h || !net || !v || !z) return PN_ERR_ARG;
    if (h->dims != 3 || h->periodic)
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_cnn_precondition: 3D vacuum-boundary handles only");
    if (h->R % 8) return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_cnn_precondition: R must be a multiple of 8");
    const int64_t V = int64_t(h->R) * h->R * h->R;
    float* scratch = nullptr;
    if (cudaMalloc(&scratch, size_t(V) * (2 * h->K + 3) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return pn_fail(h, PN_ERR_ALLOC, "pn_cnn_precondition: scratch");
    }
    const int rc = pn::precond_apply(h, net, v, z, scratch, h->d_scalars + 100, (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(scratch);
    return rc;
}

}  // extern "C"
