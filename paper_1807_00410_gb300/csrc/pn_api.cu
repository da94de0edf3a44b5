// C ABI of the GB300 P_N library: handles, layout, medium upload and the
// operator / vector entry points.  The solver entry point is in pn_solve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pn_internal.h"

static std::string g_create_error;

int pn_fail(pn_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int pn_cuda_fail(pn_handle* h, cudaError_t e, const char* where) {
    return pn_fail(h, PN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int pn_sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (dev >= 0 && dev < kMaxDev) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    } else if (dev >= 0 && dev < kMaxDev) {
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t pn_smem_attr_once(std::atomic<unsigned long long>& done, const void* func, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

namespace {

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Copy n elements of a host or device array of PN_F32/PN_F64 into a host
// double vector.
int load_field(pn_handle* h, const void* src, int64_t n, int dtype, int on_device, std::vector<double>& out) {
    out.resize(size_t(n));
    const size_t esz = dtype == PN_F32 ? 4 : 8;
    std::vector<unsigned char> tmp;
    const void* hp = src;
    if (on_device) {
        tmp.resize(size_t(n) * esz);
        cudaError_t e = cudaMemcpy(tmp.data(), src, size_t(n) * esz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_create: reading medium");
        hp = tmp.data();
    }
    if (dtype == PN_F32) {
        const float* f = (const float*)hp;
        for (int64_t i = 0; i < n; ++i) out[size_t(i)] = f[i];
    } else {
        std::memcpy(out.data(), hp, size_t(n) * 8);
    }
    return PN_OK;
}

template <typename T>
int dev_alloc(pn_handle* h, T** p, size_t count, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return pn_fail(h, PN_ERR_ALLOC, std::string("pn_create: cudaMalloc failed for ") + what);
    }
    return PN_OK;
}

// Writes one padded plane from a voxel-centre field: every active slot gets
// the mean of its adjacent in-domain centres, every other slot 0.
__global__ void k_fill_plane(const double* F, int R, int px, int py, int pz, int64_t pitch_x,
                             int64_t pitch_y, int64_t nzb, int64_t plane_stride, int periodic, double* out_d,
                             float* out_f) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < plane_stride;
         s += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(s % pitch_x);
        const int64_t t = s / pitch_x;
        const int y = int(t % (R + 1));
        const int z = int(t / (R + 1));
        double v = 0.0;
        const int ext = periodic ? 0 : 1;
        if (s < pitch_y * nzb && x < R + ext * px && y < R + ext * py && z < R + ext * pz) {
            // in-domain centres adjacent to the slot (periodic: face i between centres i - 1 mod R and i)
            int x0 = px ? max(x - 1, 0) : x, x1 = px ? min(x, R - 1) : x;
            int y0 = py ? max(y - 1, 0) : y, y1 = py ? min(y, R - 1) : y;
            int z0 = pz ? max(z - 1, 0) : z, z1 = pz ? min(z, R - 1) : z;
            if (periodic) {
                x0 = px ? (x + R - 1) % R : x;
                y0 = py ? (y + R - 1) % R : y;
                z0 = pz ? (z + R - 1) % R : z;
                x1 = x;
                y1 = y;
                z1 = z;
            }
            const int64_t R2 = int64_t(R) * R;
            v = 0.125 * (F[z0 * R2 + y0 * R + x0] + F[z0 * R2 + y0 * R + x1] + F[z0 * R2 + y1 * R + x0] +
                         F[z0 * R2 + y1 * R + x1] + F[z1 * R2 + y0 * R + x0] + F[z1 * R2 + y0 * R + x1] +
                         F[z1 * R2 + y1 * R + x0] + F[z1 * R2 + y1 * R + x1]);
        }
        out_d[s] = v;
        out_f[s] = float(v);
    }
}

void free_all(pn_handle* h) {
    void* ptrs[] = {h->d_planes, h->d_terms, h->d_st_f, h->d_ss_f, h->d_st_d, h->d_ss_d,
                    h->d_q_f,    h->d_q_d,   h->d_partials, h->d_scalars, h->d_work, h->d_ir, h->d_cmean};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    h->prof_ev.clear();
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->side = nullptr;
    h->ev_fork = h->ev_join = nullptr;
    if (h->solve_s) cudaStreamDestroy(h->solve_s);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    h->solve_s = nullptr;
    h->ev_in = h->ev_out = nullptr;
}

}  // namespace

void pn_prof_reset(pn_handle* h, bool on) {
    h->prof_on = on;
    h->prof_pending.clear();
    for (int k = 0; k < PN_PROF_KINDS; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
        h->prof_bytes[k] = 0.0;
    }
}

void pn_prof_begin(pn_handle* h, cudaStream_t s) {
    if (!h->prof_on) return;
    const size_t need = 2 * (h->prof_pending.size() + 1);
    while (h->prof_ev.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            h->prof_on = false;  // out of events: stop profiling, keep solving
            cudaGetLastError();
            return;
        }
        h->prof_ev.push_back(e);
    }
    cudaEventRecord(h->prof_ev[need - 2], s);
}

void pn_prof_end(pn_handle* h, cudaStream_t s, int kind, double bytes) {
    if (!h->prof_on) return;
    const size_t i = 2 * h->prof_pending.size();
    if (i + 1 >= h->prof_ev.size()) return;
    cudaEventRecord(h->prof_ev[i + 1], s);
    h->prof_pending.emplace_back(kind, bytes);
}

void pn_prof_drain(pn_handle* h) {
    for (size_t i = 0; i < h->prof_pending.size(); ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const int k = h->prof_pending[i].first;
        h->prof_ms[k] += ms;
        h->prof_n[k] += 1;
        h->prof_bytes[k] += h->prof_pending[i].second;
    }
    h->prof_pending.clear();
}

extern "C" {

int pn_profile_get(const pn_handle* h, int kind, double* ms, int64_t* launches, double* bytes) {
    if (!h || kind < 0 || kind >= PN_PROF_KINDS) return PN_ERR_ARG;
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_n[kind];
    if (bytes) *bytes = h->prof_bytes[kind];
    return PN_OK;
}

const char* pn_last_error(const pn_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void pn_default_solve_opts(pn_solve_opts* o) {
    if (!o) return;
    o->solver = PN_SOLVER_CGLS;
    o->precision = PN_F64;
    o->tol = 1e-6;
    o->max_iter = 100000;
    o->restart = 60;
    o->inner_tol = 1e-2;
    o->max_outer = 50;
    o->check_every = 10;
    o->profile = 0;
    o->ortho = PN_ORTHO_CGS2;
    o->precond = nullptr;
    o->basis = PN_BASIS_F32;
    o->augment = 0;
}

}  // extern "C"

namespace {

// pn_create (dims 3) and pn_create_2d (dims 2, the z-independent reduction:
// coefficients with l + m even, x and y transport only, R^2 centre fields).
int create_impl(pn_handle** out, int N, int R, const pn_medium* m, int boundary, void* stream, int dims) {
    if (!out) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: out is NULL");
    *out = nullptr;
    if (N < 0 || N > PN_MAX_N) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: N must be in [0, 7]");
    if (R < 2 || R > (dims == 3 ? 1024 : 16384))
        return pn_fail(nullptr, PN_ERR_ARG, dims == 3 ? "pn_create: R must be in [2, 1024]"
                                                      : "pn_create_2d: R must be in [2, 16384]");
    if (!m || !m->sigma_t) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: medium or sigma_t is NULL");
    if (m->dtype != PN_F32 && m->dtype != PN_F64) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: bad medium dtype");
    if (boundary != PN_BC_VACUUM && boundary != PN_BC_PERIODIC_TEST)
        return pn_fail(nullptr, PN_ERR_ARG, "pn_create: boundary must be PN_BC_VACUUM or PN_BC_PERIODIC_TEST");
    if (boundary == PN_BC_PERIODIC_TEST && dims != 3)
        return pn_fail(nullptr, PN_ERR_UNSUPPORTED, "pn_create_2d: the periodic test mode is 3D only");
    if (m->Q && m->q_mode != PN_Q_CENTRE_00 && m->q_mode != PN_Q_CENTRE_MOMENTS)
        return pn_fail(nullptr, PN_ERR_ARG, "pn_create: bad q_mode");
    if (!(std::fabs(m->g) < 1.0)) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: |g| must be < 1");
    if (!(m->sigma_t_min >= 0.0)) return pn_fail(nullptr, PN_ERR_ARG, "pn_create: sigma_t_min must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;

    pn_handle* h = new (std::nothrow) pn_handle();
    if (!h) return pn_fail(nullptr, PN_ERR_ALLOC, "pn_create: host allocation failed");
    cudaGetDevice(&h->device);
    h->N = N;
    h->dims = dims;
    h->periodic = boundary == PN_BC_PERIODIC_TEST ? 1 : 0;
    h->R = R;
    h->h = 1.0 / R;
    h->g = m->g;
    h->pitch_x = round_up(R + 1, 4);
    h->pitch_y = h->pitch_x * (R + 1);
    h->nz_box = dims == 3 ? R + 1 : 1;
    h->plane_stride = round_up(h->pitch_y * h->nz_box, 32);

    // planes grouped by parity class, coefficient order within a class; the
    // 2D reduction keeps the classes with pz = 0 (l + m even)
    const int K3 = (N + 1) * (N + 1);
    std::vector<int> cls_of_k(K3), idx2(K3, -1);
    for (int l = 0, k = 0; l <= N; ++l)
        for (int mm = -l; mm <= l; ++mm, ++k) {
            int px, py, pz;
            pn::parity_bits(l, mm, px, py, pz);
            cls_of_k[k] = px + 2 * py + 4 * pz;
        }
    for (int k = 0, j = 0; k < K3; ++k)
        if (cls_of_k[k] < 4) idx2[k] = j++;  // position in the 2D coefficient list
    for (int q = 0; q < PN_MAX_K; ++q) h->plane_k[q] = h->plane_class[q] = h->plane_of_k[q] = -1;
    int p = 0;
    for (int c = 0; c < (dims == 3 ? 8 : 4); ++c)
        for (int k = 0; k < K3; ++k)
            if (cls_of_k[k] == c) {
                h->plane_k[p] = k;
                h->plane_class[p] = c;
                h->plane_of_k[k] = p;
                ++p;
            }
    h->K = p;
    h->n_elems = h->plane_stride * h->K;
    const int K = h->K;

    std::vector<double> A;
    pn::transport_couplings(N, A);
    h->planes.resize(K);
    h->n_active = 0;
    for (int q = 0; q < K; ++q) {
        const int k = h->plane_k[q];
        int l = 0;
        while ((l + 1) * (l + 1) <= k) ++l;
        pn::Plane P;
        P.k = k;
        P.l = l;
        P.m = k - l * l - l;
        P.kc = dims == 3 ? k : idx2[k];
        P.cls = h->plane_class[q];
        P.px = P.cls & 1;
        P.py = (P.cls >> 1) & 1;
        P.pz = (P.cls >> 2) & 1;
        P.fl_d = l == 0 ? 1.0 : std::pow(m->g, l);
        P.fl_f = float(P.fl_d);
        P.t0 = int(h->terms.size());
        for (int d = 0; d < dims; ++d)
            for (int kp = 0; kp < K3; ++kp) {
                const double a = A[(size_t(d) * K3 + k) * K3 + kp];
                if (a == 0.0) continue;
                pn::Term t;
                t.q = h->plane_of_k[kp];
                if (t.q < 0) {  // A_x, A_y never couple l + m even to odd: unreachable
                    delete h;
                    return pn_fail(nullptr, PN_ERR_ARG, "pn_create: coupling to a coefficient outside the layout");
                }
                t.axis = d;
                t.cd = a * R;  // A_d / h
                t.cf = float(t.cd);
                h->terms.push_back(t);
            }
        P.t1 = int(h->terms.size());
        h->planes[q] = P;
        const int ext = h->periodic ? 0 : 1;
        h->n_active += int64_t(R + ext * P.px) * (R + ext * P.py) * (dims == 3 ? R + ext * P.pz : 1);
    }

    int rc = PN_OK;
    const int64_t V = dims == 3 ? int64_t(R) * R * R : int64_t(R) * R;
    std::vector<double> st, al;
#define PN_TRY(x)                       \
    do {                                \
        rc = (x);                       \
        if (rc != PN_OK) goto fail;     \
    } while (0)
    PN_TRY(load_field(nullptr, m->sigma_t, V, m->dtype, m->on_device, st));
    if (m->albedo) PN_TRY(load_field(nullptr, m->albedo, V, m->dtype, m->on_device, al));
    {
        std::vector<double> ss(static_cast<size_t>(V));
        std::vector<float> stf(static_cast<size_t>(V)), ssf(static_cast<size_t>(V));
        for (int64_t i = 0; i < V; ++i) {
            double t = st[size_t(i)];
            if (!std::isfinite(t)) {
                rc = pn_fail(nullptr, PN_ERR_ARG, "pn_create: non-finite sigma_t");
                goto fail;
            }
            t = std::max(t, m->sigma_t_min);
            const double a = m->albedo ? al[size_t(i)] : m->albedo_const;
            if (!std::isfinite(a)) {
                rc = pn_fail(nullptr, PN_ERR_ARG, "pn_create: non-finite albedo");
                goto fail;
            }
            st[size_t(i)] = t;
            ss[size_t(i)] = a * t;
            stf[size_t(i)] = float(t);
            ssf[size_t(i)] = float(a * t);
        }
        PN_TRY(dev_alloc(nullptr, &h->d_st_d, size_t(V), "sigma_t"));
        PN_TRY(dev_alloc(nullptr, &h->d_ss_d, size_t(V), "sigma_s"));
        PN_TRY(dev_alloc(nullptr, &h->d_st_f, size_t(V), "sigma_t"));
        PN_TRY(dev_alloc(nullptr, &h->d_ss_f, size_t(V), "sigma_s"));
        cudaError_t e = cudaMemcpy(h->d_st_d, st.data(), V * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_ss_d, ss.data(), V * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_st_f, stf.data(), V * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_ss_f, ssf.data(), V * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create: uploading medium");
            goto fail;
        }
    }
    PN_TRY(dev_alloc(nullptr, &h->d_planes, size_t(K), "planes"));
    PN_TRY(dev_alloc(nullptr, &h->d_terms, std::max<size_t>(1, h->terms.size()), "terms"));
    {
        cudaError_t e = cudaMemcpy(h->d_planes, h->planes.data(), K * sizeof(pn::Plane), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !h->terms.empty())
            e = cudaMemcpy(h->d_terms, h->terms.data(), h->terms.size() * sizeof(pn::Term), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create: uploading tables");
            goto fail;
        }
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create: side stream");
            goto fail;
        }
    }
    // scratch
    h->red_blocks = pn::reduce_blocks();
    PN_TRY(dev_alloc(nullptr, &h->d_partials,
                     size_t(std::max(std::max(h->red_blocks, 8 * pn_sm_count()) * (PN_MAX_MDOT + 1),
                                             std::max(h->dims == 3 ? pn::tiled_partial_bound(h) : 0,
                                                      std::max(pn::op_partial_count(h, PN_F32),
                                                               pn::op_partial_count(h, PN_F64))))),
                     "partials"));
    PN_TRY(dev_alloc(nullptr, &h->d_scalars, size_t(PN_NSCALARS), "scalars"));
    {
        const cudaError_t e = cudaMemset(h->d_scalars, 0, size_t(PN_NSCALARS) * sizeof(double));
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create: scalars");
            goto fail;
        }
    }
    if (cudaMallocHost((void**)&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) {
        h->h_pinned = nullptr;
        rc = pn_fail(nullptr, PN_ERR_ALLOC, "pn_create: pinned host allocation failed");
        goto fail;
    }
    // source
    h->n_q_planes = !m->Q ? 0 : (m->q_mode == PN_Q_CENTRE_00 ? 1 : K);
    if (h->n_q_planes > 0) {
        PN_TRY(dev_alloc(nullptr, &h->d_q_d, size_t(h->n_q_planes) * h->plane_stride, "Q"));
        PN_TRY(dev_alloc(nullptr, &h->d_q_f, size_t(h->n_q_planes) * h->plane_stride, "Q"));
        double* tmp = nullptr;
        PN_TRY(dev_alloc(nullptr, &tmp, size_t(V), "Q staging"));
        std::vector<double> qk;
        const unsigned char* base = (const unsigned char*)m->Q;
        const size_t esz = m->dtype == PN_F32 ? 4 : 8;
        for (int q = 0; q < h->n_q_planes && rc == PN_OK; ++q) {
            // q_mode 0: plane 0 is coefficient 0 (class 0 comes first); in 2D
            // the moments come in the order of the 2D coefficient list
            const int k = h->n_q_planes == 1 ? 0 : (dims == 3 ? h->plane_k[q] : idx2[h->plane_k[q]]);
            rc = load_field(nullptr, base + size_t(k) * V * esz, V, m->dtype, m->on_device, qk);
            if (rc != PN_OK) break;
            cudaError_t e = cudaMemcpy(tmp, qk.data(), V * 8, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                rc = pn_cuda_fail(nullptr, e, "pn_create: uploading Q");
                break;
            }
            const pn::Plane& P = h->planes[q];
            k_fill_plane<<<8 * pn_sm_count(), 256, 0, s>>>(tmp, R, P.px, P.py, P.pz, h->pitch_x, h->pitch_y,
                                                         h->nz_box, h->plane_stride, h->periodic,
                                                         h->d_q_d + q * h->plane_stride,
                                                         h->d_q_f + q * h->plane_stride);
            e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) rc = pn_cuda_fail(nullptr, e, "pn_create: filling Q");
        }
        cudaFree(tmp);
        if (rc != PN_OK) goto fail;
        cudaError_t e = pn::launch_dot(h, h->d_q_d, h->d_q_d, int64_t(h->n_q_planes) * h->plane_stride, PN_F64,
                                       h->d_scalars, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_pinned, h->d_scalars, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create: norm of Q");
            goto fail;
        }
        h->q_norm2 = h->h_pinned[0];
    }
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = pn_cuda_fail(nullptr, e, "pn_create");
            goto fail;
        }
    }
#undef PN_TRY
    *out = h;
    return PN_OK;
fail:
    free_all(h);
    delete h;
    return rc;
}

}  // namespace

extern "C" {

int pn_create(pn_handle** out, int N, int R, const pn_medium* m, int boundary, void* stream) {
    return create_impl(out, N, R, m, boundary, stream, 3);
}

int pn_create_2d(pn_handle** out, int N, int R, const pn_medium* m, int boundary, void* stream) {
    return create_impl(out, N, R, m, boundary, stream, 2);
}

int pn_destroy(pn_handle* h) {
    if (!h) return PN_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    free_all(h);
    pn::tma_cache_free(h);
    if (dev != h->device) cudaSetDevice(dev);
    delete h;
    return PN_OK;
}

int pn_get_layout(const pn_handle* h, pn_layout_info* o) {
    if (!h || !o) return PN_ERR_ARG;
    o->N = h->N;
    o->K = h->K;
    o->R = h->R;
    o->pitch_x = h->pitch_x;
    o->pitch_y = h->pitch_y;
    o->plane_stride = h->plane_stride;
    o->n_elems = h->n_elems;
    o->n_active = h->n_active;
    for (int p = 0; p < PN_MAX_K; ++p) {
        o->plane_k[p] = h->plane_k[p];
        o->plane_class[p] = h->plane_class[p];
    }
    return PN_OK;
}

static int check_vec_args(pn_handle* h, const void* a, const void* b, int dtype, const char* fn) {
    if (!h) return PN_ERR_ARG;
    if (!a || !b) return pn_fail(h, PN_ERR_ARG, std::string(fn) + ": NULL vector");
    if (dtype != PN_F32 && dtype != PN_F64) return pn_fail(h, PN_ERR_ARG, std::string(fn) + ": bad dtype");
    if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u)
        return pn_fail(h, PN_ERR_ARG, std::string(fn) + ": vectors must be 16-byte aligned");
    return PN_OK;
}

static int run_op(pn_handle* h, int mode, const void* x, void* y, int dtype, void* stream, const char* fn) {
    int rc = check_vec_args(h, x, y, dtype, fn);
    if (rc != PN_OK) return rc;
    if (x == y) return pn_fail(h, PN_ERR_ARG, std::string(fn) + ": x and y must not alias");
    cudaError_t e = pn::launch_op(h, mode, x, y, dtype, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, fn);
    return PN_OK;
}

int pn_apply(pn_handle* h, const void* x, void* y, int dtype, void* stream) {
    return run_op(h, pn::OP_APPLY, x, y, dtype, stream, "pn_apply");
}

int pn_apply_t(pn_handle* h, const void* x, void* y, int dtype, void* stream) {
    return run_op(h, pn::OP_APPLY_T, x, y, dtype, stream, "pn_apply_t");
}

int pn_residual(pn_handle* h, const void* x, void* r, double* rel_out, int dtype, void* stream) {
    int rc = check_vec_args(h, x, r, dtype, "pn_residual");
    if (rc != PN_OK) return rc;
    if (x == r) return pn_fail(h, PN_ERR_ARG, "pn_residual: x and r must not alias");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = pn::launch_op(h, pn::OP_RESIDUAL, x, r, dtype, rel_out ? h->d_partials : nullptr, s);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_residual");
    if (rel_out) {
        e = pn::launch_reduce(h->d_partials, pn::op_partial_count(h, dtype), 1, h->d_scalars, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_pinned, h->d_scalars, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_residual");
        const double rr = h->h_pinned[0];
        *rel_out = h->q_norm2 > 0.0 ? std::sqrt(rr / h->q_norm2) : std::sqrt(rr);
        if (!std::isfinite(*rel_out)) return pn_fail(h, PN_ERR_NONFINITE, "pn_residual: non-finite residual");
    }
    return PN_OK;
}

int pn_dot(pn_handle* h, const void* x, const void* y, double* out, int dtype, void* stream) {
    int rc = check_vec_args(h, x, y, dtype, "pn_dot");
    if (rc != PN_OK) return rc;
    if (!out) return pn_fail(h, PN_ERR_ARG, "pn_dot: out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = pn::launch_dot(h, x, y, h->n_elems, dtype, h->d_scalars, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_pinned, h->d_scalars, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_dot");
    *out = h->h_pinned[0];
    return PN_OK;
}

int pn_set_apply_tiling(pn_handle* h, int ctas_per_sm) {
    if (!h) return PN_ERR_ARG;
    if (ctas_per_sm < 1 || ctas_per_sm > 16) return pn_fail(h, PN_ERR_ARG, "pn_set_apply_tiling: ctas_per_sm in [1, 16]");
    h->tile_ctas_per_sm = ctas_per_sm;
    return PN_OK;
}

int pn_get_apply_plan(const pn_handle* h, int* ctas_per_sm, int* kernel, int* face_serial) {
    if (!h) return PN_ERR_ARG;
    if (ctas_per_sm) *ctas_per_sm = h->tile_ctas_per_sm;
    if (kernel) pn_get_apply_kernel(h, kernel);
    if (face_serial) *face_serial = h->face_serial;
    return PN_OK;
}

int pn_set_stream_kernels(pn_handle* h, int tma) {
    if (!h) return PN_ERR_ARG;
    if (tma < 0 || tma > 3) return pn_fail(h, PN_ERR_ARG, "pn_set_stream_kernels: mask in [0, 3]");
    h->stream_tma = tma;
    return PN_OK;
}

int pn_set_pdl(pn_handle* h, int on) {
    if (!h) return PN_ERR_ARG;
    h->pdl_enabled = on ? 1 : 0;
    return PN_OK;
}

int pn_set_l2_residency(pn_handle* h, int on) {
    if (!h) return PN_ERR_ARG;
    h->l2_resident = on ? 1 : 0;
    return PN_OK;
}

int pn_set_apply_kernel(pn_handle* h, int kernel) {
    if (!h) return PN_ERR_ARG;
    if (kernel != PN_APPLY_KERNEL_REGISTER && kernel != PN_APPLY_KERNEL_TMA)
        return pn_fail(h, PN_ERR_ARG, "pn_set_apply_kernel: bad kernel");
    if (kernel == PN_APPLY_KERNEL_TMA && pn::tiled_serves(h) && !pn::tma_serves(h))
        return pn_fail(h, PN_ERR_UNSUPPORTED, "pn_set_apply_kernel: the TMA kernel does not serve this handle");
    h->tile_kernel = kernel;
    return PN_OK;
}

int pn_get_apply_kernel(const pn_handle* h, int* kernel) {
    if (!h || !kernel) return PN_ERR_ARG;
    *kernel = (h->tile_kernel == PN_APPLY_KERNEL_TMA && pn::tma_serves(h)) ? PN_APPLY_KERNEL_TMA
                                                                             : PN_APPLY_KERNEL_REGISTER;
    return PN_OK;
}

int pn_tune_apply(pn_handle* h, void* stream, int* ctas_per_sm, double* best_ms) {
    if (!h) return PN_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* x = nullptr;
    float* y = nullptr;
    if (cudaMalloc(&x, size_t(h->n_elems) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&y, size_t(h->n_elems) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (x) cudaFree(x);
        return pn_fail(h, PN_ERR_ALLOC, "pn_tune_apply: vectors");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(x, 0, size_t(h->n_elems) * sizeof(float), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int cands[] = {1, 2, 4, 8};
    int best = h->tile_ctas_per_sm, best_k = h->tile_kernel, best_f = h->face_serial;
    float best_t = 1e30f, best_raw = 0.0f;
    const int nk = pn::tma_serves(h) ? 2 : 1;
    // With programmatic dependent launch enabled (the solvers' Arnoldi steps)
    // each timing is a chain of kChain applies launched the way the solver
    // launches them (face-column kernel first, the main kernel overlapping
    // it): a plan that wins in isolation can lose there (P5 64^3: 1 CTA per
    // SM 36.8 against 38.0 us alone, 83.9 against 78.2 ms per solve).
    const bool chain = h->pdl_enabled != 0;
    constexpr int kChain = 4;
    for (int ci = 0; ci < 8 * nk; ++ci) {
        const int c = cands[ci % 4];
        if (e != cudaSuccess) break;
        h->tile_ctas_per_sm = c;
        h->face_serial = (ci / 4) % 2;
        h->tile_kernel = nk == 2 ? ci / 8 : PN_APPLY_KERNEL_REGISTER;
        // median of 10 timed launches after 2 warm-ups; the concurrent face
        // schedule must win by 3 % (its event joins cost more inside a solve,
        // between other kernels, than in back-to-back applies)
        float t[10];
        for (int rep = 0; rep < 12 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            h->pdl = chain ? 1 : 0;
            for (int q = 0; q < (chain ? kChain : 1) && e == cudaSuccess; ++q)
                e = pn::launch_op(h, pn::OP_APPLY, x, y, PN_F32, nullptr, s);
            h->pdl = 0;
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2) t[rep - 2] = ms / float(chain ? kChain : 1);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 10);
        const float raw = 0.5f * (t[4] + t[5]);
        const float med = raw * (h->face_serial ? 1.0f : 1.03f);
        if (med < best_t) {
            best_t = med;
            best_raw = raw;
            best = c;
            best_k = h->tile_kernel;
            best_f = h->face_serial;
        }
    }
    h->tile_ctas_per_sm = best;
    h->tile_kernel = best_k;
    h->face_serial = best_f;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_tune_apply");
    if (ctas_per_sm) *ctas_per_sm = best;
    if (best_ms) *best_ms = best_raw;
    return PN_OK;
}

int pn_axpby(pn_handle* h, double alpha, const void* x, double beta, void* y, int dtype, void* stream) {
    int rc = check_vec_args(h, x, y, dtype, "pn_axpby");
    if (rc != PN_OK) return rc;
    cudaError_t e = pn::launch_axpby(h->n_elems, alpha, x, beta, y, dtype, (cudaStream_t)stream);
    if (e != cudaSuccess) return pn_cuda_fail(h, e, "pn_axpby");
    return PN_OK;
}

}  // extern "C"
