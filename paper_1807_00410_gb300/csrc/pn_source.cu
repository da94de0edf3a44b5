// Source building and unstaggering (the paper's section "Rendering").
//
// pn_single_scatter_beam: the single-scattered light of a collimated beam
// folded into the emission term, Q^{l,m}(x) = sigma_s(x) E(x) g^l Y_{l,m}(w_b)
// (Funk-Hecke projection of sigma_s int p(w'->w) L_u(w') dw' with the
// uncollided light L_u = E(x) delta(w' - w_b), E = exp(-int sigma_t ds)).
// One thread per transverse line marches along the beam, accumulating the
// optical depth (whole cells before the voxel plus half of its own).
//
// pn_unstagger: every coefficient interpolated to voxel centres (the mean of
// the two faces of the cell along each axis on which it lives on faces).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "pn_internal.h"

namespace {

// Real spherical harmonic with the Condon-Shortley phase (the basis the
// printed P_N equations are written in), evaluated on the host.
double assoc_legendre(int l, int m, double x) {  // without the (-1)^m phase
    const double s = std::sqrt(std::fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2 * i - 1) * s;
    if (l == m) return pmm;
    double pm1 = x * (2 * m + 1) * pmm;
    if (l == m + 1) return pm1;
    double a = pmm, b = pm1;
    for (int ll = m + 2; ll <= l; ++ll) {
        const double c = ((2 * ll - 1) * x * b - (ll + m - 1) * a) / (ll - m);
        a = b;
        b = c;
    }
    return b;
}

double real_sh(int l, int m, double theta, double phi) {
    const int am = m < 0 ? -m : m;
    double fact = 1.0;  // (l - |m|)! / (l + |m|)!
    for (int i = l - am + 1; i <= l + am; ++i) fact /= i;
    const double nlm = std::sqrt((2 * l + 1) / (4.0 * M_PI) * fact);
    const double p = assoc_legendre(l, am, std::cos(theta));
    if (m == 0) return nlm * p;
    const double sgn = (am & 1) ? -1.0 : 1.0;
    const double ang = m > 0 ? std::cos(am * phi) : std::sin(am * phi);
    return sgn * std::sqrt(2.0) * nlm * p * ang;
}

template <typename T>
struct BeamArgs {
    const T* st;
    const T* albedo;   // or null
    double albedo_const;
    T* q;              // K x R^3
    int R, K, axis, sign;
    double radius2, c0, c1;
    double coef[PN_MAX_K];  // g^l Y_{l,m}(w_b) per coefficient k
};

template <typename T>
__global__ void k_beam(BeamArgs<T> a) {
    const int R = a.R;
    const int64_t line = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (line >= int64_t(R) * R) return;
    const int u = int(line % R), v = int(line / R);  // transverse indices (lower axis first)
    const double h = 1.0 / R;
    const double tu = (u + 0.5) * h - a.c0, tv = (v + 0.5) * h - a.c1;
    const bool inside = tu * tu + tv * tv <= a.radius2;
    // strides of the beam axis and of the two transverse axes in [z][y][x]
    const int64_t sx = 1, sy = R, sz = int64_t(R) * R;
    int64_t s_ax, s_u, s_v;
    if (a.axis == 0) { s_ax = sx; s_u = sy; s_v = sz; }
    else if (a.axis == 1) { s_ax = sy; s_u = sx; s_v = sz; }
    else { s_ax = sz; s_u = sx; s_v = sy; }
    const int64_t base = u * s_u + v * s_v;
    const int64_t V = int64_t(R) * R * R;
    double tau = 0.0;
    for (int t = 0; t < R; ++t) {
        const int i = a.sign > 0 ? t : R - 1 - t;
        const int64_t idx = base + i * s_ax;
        const double st = double(a.st[idx]);
        const double E = inside ? exp(-(tau + 0.5 * st * h)) : 0.0;
        tau += st * h;
        const double ss = st * (a.albedo ? double(a.albedo[idx]) : a.albedo_const);
        for (int k = 0; k < a.K; ++k) a.q[k * V + idx] = T(ss * E * a.coef[k]);
    }
}

template <typename T>
__global__ void k_unstagger(const T* x, T* out, const pn::Plane* planes, int R, int nzc, int64_t pitch_x,
                            int64_t pitch_y, int64_t plane_stride, int K) {
    const int64_t V = int64_t(R) * R * nzc;  // cells (nzc = R; 1 for the 2D reduction, whose planes have pz = 0)
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < V * K; t += int64_t(gridDim.x) * blockDim.x) {
        const int p = int(t / V);
        const int64_t c = t % V;
        const int xi = int(c % R), yi = int((c / R) % R), zi = int(c / (int64_t(R) * R));
        const pn::Plane P = planes[p];
        const T* b = x + int64_t(p) * plane_stride;
        T acc = T(0);
        for (int dz = 0; dz <= P.pz; ++dz)
            for (int dy = 0; dy <= P.py; ++dy)
                for (int dx = 0; dx <= P.px; ++dx)
                    acc += b[(zi + dz) * pitch_y + (yi + dy) * pitch_x + xi + dx];
        const int n = (1 + P.px) * (1 + P.py) * (1 + P.pz);
        out[int64_t(P.kc) * V + c] = acc / T(n);
    }
}

}  // namespace

extern "C" int pn_single_scatter_beam(int N, int R, const void* sigma_t, const void* albedo, double albedo_const,
                                      double g, int axis, int sign, double radius, double c0, double c1, void* Q,
                                      int dtype, void* stream) {
    if (N < 0 || N > PN_MAX_N || R < 1 || R > 1024 || !sigma_t || !Q) return PN_ERR_ARG;
    if (axis < 0 || axis > 2 || (sign != 1 && sign != -1) || !(radius >= 0.0) || !(std::fabs(g) < 1.0))
        return PN_ERR_ARG;
    if (dtype != PN_F32 && dtype != PN_F64) return PN_ERR_ARG;
    const double pi = M_PI;
    double theta = axis == 2 ? 0.0 : 0.5 * pi, phi = axis == 1 ? 0.5 * pi : 0.0;
    if (sign < 0) {
        theta = pi - theta;
        phi += pi;
    }
    const int K = (N + 1) * (N + 1);
    const int blocks = int((int64_t(R) * R + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    auto fill = [&](auto* args) {
        args->R = R;
        args->K = K;
        args->axis = axis;
        args->sign = sign;
        args->radius2 = radius * radius;
        args->c0 = c0;
        args->c1 = c1;
        args->albedo_const = albedo_const;
        for (int l = 0, k = 0; l <= N; ++l)
            for (int m = -l; m <= l; ++m, ++k) args->coef[k] = (l == 0 ? 1.0 : std::pow(g, l)) * real_sh(l, m, theta, phi);
    };
    if (dtype == PN_F32) {
        BeamArgs<float> a{};
        fill(&a);
        a.st = (const float*)sigma_t;
        a.albedo = (const float*)albedo;
        a.q = (float*)Q;
        k_beam<float><<<blocks, 256, 0, s>>>(a);
    } else {
        BeamArgs<double> a{};
        fill(&a);
        a.st = (const double*)sigma_t;
        a.albedo = (const double*)albedo;
        a.q = (double*)Q;
        k_beam<double><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? PN_OK : PN_ERR_CUDA;
}

extern "C" int pn_unstagger(pn_handle* h, const void* x, void* out, int dtype, void* stream) {
    if (!h) return PN_ERR_ARG;
    if (!x || !out || (dtype != PN_F32 && dtype != PN_F64)) return pn_fail(h, PN_ERR_ARG, "pn_unstagger: bad argument");
    if (h->periodic) return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_unstagger: not in the periodic test mode");
    const int nzc = h->dims == 3 ? h->R : 1;
    const int64_t V = int64_t(h->R) * h->R * nzc;
    const int blocks = int(std::min<int64_t>((V * h->K + 255) / 256, 8 * int64_t(pn_sm_count()) * 8));
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == PN_F32)
        k_unstagger<float><<<blocks, 256, 0, s>>>((const float*)x, (float*)out, h->d_planes, h->R, nzc, h->pitch_x,
                                                  h->pitch_y, h->plane_stride, h->K);
    else
        k_unstagger<double><<<blocks, 256, 0, s>>>((const double*)x, (double*)out, h->d_planes, h->R, nzc,
                                                   h->pitch_x, h->pitch_y, h->plane_stride, h->K);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_unstagger");
    return PN_OK;
}
