// Internal declarations of the GB300 P_N library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "pn_gb300.h"

namespace pn {

// One transport coupling of an output plane:
//   y_p(s) += c * (x_q(s + (1 - b) e_axis) - x_q(s - b e_axis)),   c = A_d[k_p, k_q] / h
// where b is plane p's parity bit along `axis` (slot arithmetic of the layout).
struct Term {
    int q;       // input plane
    int axis;    // 0 = x, 1 = y, 2 = z
    float cf;    // c in FP32
    double cd;   // c in FP64
};

// Per-plane description.
struct Plane {
    int k, l, m;       // coefficient (k = l^2 + l + m)
    int kc;            // its index in the handle's coefficient list (3D: k; 2D: among l + m even)
    int cls;           // px + 2 py + 4 pz
    int px, py, pz;    // parity bits
    int t0, t1;        // term range [t0, t1) in the term table
    float fl_f;        // scattering factor g^l
    double fl_d;
};

// Angular transport couplings from the closed forms of the appendix's final
// real P_N equations.  A[d][k][k'] dense, d = x, y, z.  Defined in pn_tables.cpp.
void transport_couplings(int N, std::vector<double>& A /* 3*K*K */);

// Parity class bits of coefficient (l, m).
inline void parity_bits(int l, int m, int& px, int& py, int& pz) {
    int am = m < 0 ? -m : m;
    px = m >= 0 ? (m & 1) : ((am + 1) & 1);
    py = m < 0 ? 1 : 0;
    pz = (l + am) & 1;
}

}  // namespace pn

// Number of SMs of the current device (cached per device ordinal).
int pn_sm_count();

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device: bit d of *done records that device d has it (the
// attribute belongs to the device context, so every device needs its own
// call).  Two host threads may both make the call; it is idempotent.
cudaError_t pn_smem_attr_once(std::atomic<unsigned long long>& done, const void* func, int bytes);

struct pn_handle {
    int N = 0, K = 0, R = 0;
    int dims = 3;        // 3: R^3 cells; 2: the z-independent reduction on R^2 cells
    int periodic = 0;    // PN_BC_PERIODIC_TEST: every axis wraps, R slots per axis for every class
    int tile_ctas_per_sm = 4;  // z-chunking target of the tiled FP32 operator (pn_tune_apply)
    int tile_kernel = PN_APPLY_KERNEL_TMA;  // main kernel of the tiled operator (pn_set_apply_kernel)
    int face_serial = 0;  // face-column kernel after the main kernel on its stream (1) or concurrent (0)
    void* tma_cache = nullptr;  // tensor maps of recent input vectors (pn_apply_tma.cu)
    // the face-column kernel of the tiled operator runs on a side stream,
    // concurrently with the tiled kernel (fork / join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pn_solve runs on this stream (joined to the caller's stream by events on
    // entry and exit), which carries the L2 access-policy window of the FP16-
    // basis GMRES (pn_set_l2_residency)
    cudaStream_t solve_s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int l2_resident = 1;
    int stream_tma = 3;  // FP16-basis GMRES: bulk-copy (TMA) staged multi-dot (bit 0) and multi-axpy (bit 1)
    // set by the FP16-basis GMRES around its Arnoldi-step operator launches:
    // the tiled operator's kernels are launched with programmatic dependent
    // launch (pn_pdl.cuh), overlapping their start with the previous kernel's
    // tail; pn_set_pdl turns it off (default on)
    int pdl = 0;
    int pdl_enabled = 1;
    int64_t nz_box = 0;  // z-slices of a plane box: R + 1 (3D) or 1 (2D)
    double h = 0.0;
    double g = 0.0;  // Henyey-Greenstein mean cosine
    int64_t pitch_x = 0, pitch_y = 0, plane_stride = 0, n_elems = 0, n_active = 0;
    int plane_k[PN_MAX_K];
    int plane_class[PN_MAX_K];
    int plane_of_k[PN_MAX_K];
    std::vector<pn::Plane> planes;
    std::vector<pn::Term> terms;
    int device = 0;

    // device copies of the tables
    pn::Plane* d_planes = nullptr;
    pn::Term* d_terms = nullptr;
    // voxel-centre fields (clamped sigma_t, sigma_s = albedo sigma_t), R^3 (2D: R^2) each
    float* d_st_f = nullptr;
    float* d_ss_f = nullptr;
    double* d_st_d = nullptr;
    double* d_ss_d = nullptr;
    // source in the padded layout: n_q_planes planes (1: only Q^{0,0}, K: all)
    int n_q_planes = 0;
    float* d_q_f = nullptr;
    double* d_q_d = nullptr;
    double q_norm2 = 0.0;  // ||Q||^2 (FP64)

    // scratch: FP64 reduction partials and device scalars
    int red_blocks = 0;           // blocks of every reduction kernel
    double* d_partials = nullptr; // >= red_blocks * (PN_MAX_MDOT + 1) doubles
    double* d_scalars = nullptr;  // PN_NSCALARS doubles
    double* h_pinned = nullptr;   // pinned host mirror of a few scalars

    // Krylov workspace (lazily grown)
    void* d_work = nullptr;
    size_t work_bytes = 0;
    // iterative refinement's vectors (FP64 residual, FP32 right-hand side and
    // correction) and the LGMRES correction ring: allocated by the first solve
    // that needs them, grown on demand, kept until pn_destroy, so that later
    // solves allocate nothing
    void* d_ir = nullptr;
    size_t ir_bytes = 0;
    int64_t work_allocs = 0;  // device allocations made for d_work and d_ir so far (pn_get_workspace)
    // FP64 operator: per parity class the means of sigma_t and sigma_s over the
    // voxel centres adjacent to each slot (16 planes; built on first use)
    double* d_cmean = nullptr;

    // launch profiler of pn_solve (opts.profile): event pairs pending readout
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<std::pair<int, double>> prof_pending;
    double prof_ms[PN_PROF_KINDS] = {};
    int64_t prof_n[PN_PROF_KINDS] = {};
    double prof_bytes[PN_PROF_KINDS] = {};

    std::string err;
};

#define PN_MAX_MDOT 16
#define PN_NSCALARS 1024
// d_scalars[PN_S_FAULT] (as unsigned int): set by a kernel whose bounded wait
// ran out (the TMA-staged operator); pn_solve reports it as PN_ERR_TIMEOUT
#define PN_S_FAULT 1000

// Kernel launchers (pn_kernels.cu).  All return cudaError_t of the launch.
namespace pn {

enum OpMode { OP_APPLY = 0, OP_APPLY_T = 1, OP_RESIDUAL = 2 };

// y = op(x).  For OP_RESIDUAL y = b - A x with b = Q (bvec == null) or the
// full vector bvec and, if partials != null, the per-block FP64 sums of y^2
// go to partials[0..op_partial_count(h)).
cudaError_t launch_op(const pn_handle* h, int mode, const void* x, void* y, int dtype,
                      double* partials, cudaStream_t s, const void* bvec = nullptr);
int op_partial_count(const pn_handle* h, int dtype);
// Kernels one launch_op makes (the tiled operator: tiled + face-column kernel).
int op_launch_count(const pn_handle* h, int dtype);

// The driver's cuTensorMapEncodeTiled (pn_apply_tma.cu), or null.
void* tensor_map_encoder();

// Tiled FP32 operator (pn_apply_tiled.cu): covers x < tiled_x_end(h) of every
// plane box; one FP64 residual partial per CTA.
cudaError_t launch_tiled(const pn_handle* h, int mode, const float* x, float* y, const float* bvec,
                         double* partials, cudaStream_t s);
// The same with a device flag: the launch does nothing while *live == 0 (for
// launches recorded once into a CUDA graph and replayed while instances finish).
cudaError_t launch_tiled_gated(const pn_handle* h, int mode, const float* x, float* y, const float* bvec,
                               double* partials, const int* live, cudaStream_t s);
// Whether the tiled FP32 operator serves this handle.
bool tiled_serves(const pn_handle* h);
// Whether its TMA-staged main kernel can (pn_apply_tma.cu); the handle's cache
// of tensor maps is freed by tma_cache_free.
bool tma_serves(const pn_handle* h);
void tma_cache_free(pn_handle* h);
int tiled_partial_count(const pn_handle* h);
int tiled_partial_bound(const pn_handle* h);  // over every z-chunking pn_tune_apply may choose
int tiled_x_end(const pn_handle* h);

// partials[b] = per-block sum of a_i * b_i (FP64); then *out = sum of partials.
cudaError_t launch_dot(const pn_handle* h, const void* a, const void* b, int64_t n, int dtype,
                       double* out_dev, cudaStream_t s);
cudaError_t launch_reduce(const double* partials, int nblocks, int nvals, double* out_dev,
                          cudaStream_t s);
cudaError_t launch_axpby(int64_t n, double alpha, const void* x, double beta, void* y, int dtype,
                         cudaStream_t s);
int reduce_blocks();

}  // namespace pn

namespace pn {
// z = M(v), the learned preconditioner (pn_precond.cu); scratch: R^3 (2K+3) floats.
int precond_apply(pn_handle* h, struct pn_cnn* net, const float* v, float* z, float* scratch, double* nrm2_dev,
                  cudaStream_t s);
}

// Profiler helpers (pn_api.cu).  prof_begin/prof_end bracket one launch on
// stream s; prof_drain reads out completed pairs (call after a sync).
void pn_prof_begin(pn_handle* h, cudaStream_t s);
void pn_prof_end(pn_handle* h, cudaStream_t s, int kind, double bytes);
void pn_prof_drain(pn_handle* h);
void pn_prof_reset(pn_handle* h, bool on);

// Set the handle's error message and return code.
int pn_fail(pn_handle* h, int code, const std::string& msg);
int pn_cuda_fail(pn_handle* h, cudaError_t e, const char* where);
