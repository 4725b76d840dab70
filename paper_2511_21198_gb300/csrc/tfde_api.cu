// extern "C" entry points of libtfde (declared and documented in include/tfde.h).
#include <cmath>
#include <string>

#include "tfde_internal.h"
#include "tfde_stats.h"

namespace tfde {

cudaStream_t capture_stream() {
    constexpr int kMaxDev = 64;
    thread_local cudaStream_t cs[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    if (!cs[dev] && cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cs[dev] = nullptr;
    }
    return cs[dev];
}
const char* last_error_text();
int assemble_problem(const tfde_params*, int, cudaStream_t, tfde_problem**);
int batch_create(const tfde_params*, int, int, cudaStream_t, tfde_batch**);
namespace cnn {
int cnn_create(const int n[3], tfde_cnn** out);
int cnn_destroy(tfde_cnn* C);
int cnn_set_params(tfde_cnn* C, const float* host);
int cnn_get(const tfde_cnn* C, int what, float* host);
int cnn_predict(tfde_cnn* C, const double* u, const double* u1, const double* u2, const double* dtF,
                const double coef[9], double* x0, cudaStream_t s);
int cnn_accumulate(tfde_cnn* C, const double* u, const double* u1, const double* u2, const double* dtF,
                   const double coef[9], const double* u_next, double* loss, cudaStream_t s);
int cnn_adam(tfde_cnn* C, float lr, cudaStream_t s);
}  // namespace cnn
int batch_destroy(tfde_batch*);
int batch_cn_advance(tfde_batch*, double* const*, const double* const*, int, double, tfde_info*, cudaStream_t);
int destroy_problem(tfde_problem*);
int host_coefficients(const tfde_params*, int, double*, double*, double*, double*);
int pcg64(const tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int pgmres64(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);
int cn_drive(tfde_problem*, const double*, const double*, const double*, double*, double, tfde_info*, cudaStream_t,
             bool, const double*, int*);
// mixed path (tfde_mixed.cu)
int mixed_apply_A(const tfde_problem*, int, const double*, double*, cudaStream_t);
int mixed_apply_Pinv(const tfde_problem*, const double*, double*, cudaStream_t);
int mixed_pcg(tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int mixed_pgmres(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);
int mixed_set_device_loop(tfde_problem*, int);
int mixed_set_spectral(tfde_problem*, int);
long long mixed_graph_launches(const tfde_problem*);
int spectrum(const tfde_params*, int, const double*, tfde_spectrum_info*, cudaStream_t);
int mixed_tune(tfde_problem*, int, cudaStream_t);
int batch_tune(tfde_batch*, int, cudaStream_t);
namespace tc {
int wait_selftest(long long limit_ns, int* tmem_freed, cudaStream_t s);
int tune_export(tfde_tune_entry* out, int cap, int* count);
int tune_import(const tfde_tune_entry* in, int count);
void tune_clear();
}
}  // namespace tfde

using namespace tfde;

namespace {

// Rejects NULL and pointers the runtime reports as plain host memory.
int check_dev(const void* p, const char* name) {
    if (!p) return set_error(TFDE_EINVAL, std::string(name) + " is NULL");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TFDE_EINVAL, std::string(name) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return set_error(TFDE_EINVAL, std::string(name) + " is not device memory");
    return TFDE_OK;
}

int check_tol(double tol) {
    if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(TFDE_EINVAL, "tol must be finite and > 0");
    return TFDE_OK;
}

int pre_call() {
    // surface a pending asynchronous fault from earlier work before starting
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("pending CUDA error: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

}  // namespace

extern "C" {

int tfde_assemble(const tfde_params* params, int precision, void* stream, tfde_problem** out) {
    if (!params || !out) return set_error(TFDE_EINVAL, "NULL argument");
    *out = nullptr;
    int st = pre_call();
    if (st) return st;
    return assemble_problem(params, precision, (cudaStream_t)stream, out);
}

int tfde_destroy(tfde_problem* prob) { return destroy_problem(prob); }

int tfde_matvec(const tfde_problem* prob, int op, const double* x, double* y, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(x, "x")) || (st = check_dev(y, "y"))) return st;
    if (x == y) return set_error(TFDE_EINVAL, "x and y must not alias");
    if (op < 0 || op > 7 || ((op & TFDE_OP_STIFF) && (op & TFDE_OP_FAST)))
        return set_error(TFDE_EINVAL, "unknown op");
    if (prob->fmix) return fmix_apply_A(prob, op, x, y, (cudaStream_t)stream);
    if (prob->prec == TFDE_MIXED) return mixed_apply_A(prob, op, x, y, (cudaStream_t)stream);
    return apply_A64(prob, op & ~TFDE_OP_FAST, x, y, (cudaStream_t)stream);
}

int tfde_precond(const tfde_problem* prob, const double* r, double* z, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(r, "r")) || (st = check_dev(z, "z"))) return st;
    if (prob->fmix) return fmix_apply_Pinv(prob, r, z, (cudaStream_t)stream);
    if (prob->prec == TFDE_MIXED) return mixed_apply_Pinv(prob, r, z, (cudaStream_t)stream);
    return apply_Pinv64(prob, r, z, (cudaStream_t)stream);
}

int tfde_pcg(const tfde_problem* prob, const double* b, double* x, double tol, int maxit, tfde_info* info,
             void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(b, "b")) || (st = check_dev(x, "x")) || (st = check_tol(tol)))
        return st;
    if (b == x) return set_error(TFDE_EINVAL, "b and x must not alias");
    if (!prob->symmetric) return set_error(TFDE_EINVAL, "PCG needs k_+ = k_- on every axis");
    if (maxit < 0) return set_error(TFDE_EINVAL, "maxit must be >= 0");
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    P->chain_ok = false;
    if (prob->fmix) return fmix_pcg(P, b, x, tol, maxit, info, (cudaStream_t)stream, false);
    if (prob->prec == TFDE_MIXED) return mixed_pcg(P, b, x, tol, maxit, info, (cudaStream_t)stream, false);
    return pcg64(prob, b, x, tol, maxit, info, (cudaStream_t)stream, false);
}

int tfde_pgmres(const tfde_problem* prob, const double* b, double* x, int restart, double tol, int maxit,
                tfde_info* info, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(b, "b")) || (st = check_dev(x, "x")) || (st = check_tol(tol)))
        return st;
    if (b == x) return set_error(TFDE_EINVAL, "b and x must not alias");
    if (restart < 1 || restart > 64) return set_error(TFDE_EINVAL, "restart must lie in [1, 64]");
    if (maxit < 0) return set_error(TFDE_EINVAL, "maxit must be >= 0");
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    P->chain_ok = false;
    if (prob->fmix) return fmix_pgmres(P, b, x, restart, tol, maxit, info, (cudaStream_t)stream, false);
    if (prob->prec == TFDE_MIXED) return mixed_pgmres(P, b, x, restart, tol, maxit, info, (cudaStream_t)stream, false);
    return pgmres64(P, b, x, restart, tol, maxit, info, (cudaStream_t)stream, false);
}

int tfde_cn_step(const tfde_problem* prob, const double* u_prev, const double* F_half, const double* x0,
                 double* u_next, double tol, tfde_info* info, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(u_prev, "u_prev")) || (st = check_dev(u_next, "u_next")) ||
        (st = check_tol(tol)))
        return st;
    if (F_half && (st = check_dev(F_half, "F_half"))) return st;
    if (x0 && (st = check_dev(x0, "x0"))) return st;
    if (u_next == u_prev || u_next == F_half) return set_error(TFDE_EINVAL, "u_next aliases an input");
    if (x0 && x0 == u_prev) x0 = nullptr;
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    P->chain_ok = false;
    return cn_drive(P, u_prev, F_half, x0, u_next, tol, info, (cudaStream_t)stream, false, nullptr, nullptr);
}

int tfde_cn_advance(const tfde_problem* prob, double* u, const double* F_half, int restart, double tol,
                    tfde_info* info, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_tol(tol))) return st;
    if (F_half && (st = check_dev(F_half, "F_half"))) return st;
    if (F_half == u) return set_error(TFDE_EINVAL, "F_half aliases u");
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    const bool chained = !restart && P->chain_ok && P->chain_u == u;
    P->chain_ok = false;
    st = cn_drive(P, u, F_half, nullptr, u, tol, info, (cudaStream_t)stream, chained, nullptr, nullptr);
    if (st == TFDE_OK) {
        P->chain_ok = true;
        P->chain_u = u;
    }
    return st;
}

int tfde_cn_advance_host(const tfde_problem* prob, const double* u_host_in, double* u_host_out, double* u,
                         const double* F_half, int restart, double tol, tfde_info* info, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_tol(tol))) return st;
    if (F_half && (st = check_dev(F_half, "F_half"))) return st;
    if (F_half == u) return set_error(TFDE_EINVAL, "F_half aliases u");
    for (const void* hp : {(const void*)u_host_in, (const void*)u_host_out}) {
        if (!hp) return set_error(TFDE_EINVAL, "NULL host buffer");
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, hp) != cudaSuccess) {
            cudaGetLastError();
        } else if (at.type == cudaMemoryTypeDevice) {
            return set_error(TFDE_EINVAL, "u_host_in / u_host_out must be host memory");
        }
    }
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    const cudaStream_t s = (cudaStream_t)stream;
    auto& io = P->io;
    if (!io.stream) {
        if (cudaStreamCreateWithFlags(&io.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&io.ev_start, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&io.ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&io.ev_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&io.ev_out, cudaEventDisableTiming) != cudaSuccess)
            return set_error(TFDE_ECUDA, "creation of the copy stream failed");
        for (auto& e : io.ev_chunk)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return set_error(TFDE_ECUDA, "creation of the copy stream failed");
    }
    const size_t bytes = P->N * sizeof(double);
    io.in = u_host_in;
    io.out = u_host_out;
    io.dev = u;
    io.out_pending = io.out_valid = false;
    // u^{m-1} host -> u on the copy stream, after the work queued on `stream`
    // so far; the step waits for it only before its first read of u
    cudaEventRecord(io.ev_start, s);
    cudaStreamWaitEvent(io.stream, io.ev_start, 0);
    // large grids: in pieces, so that the right-hand-side and guess pass can
    // start on each range as it arrives (an event per piece)
    io.nchunks = P->N >= ((size_t)1 << 20) ? tfde_problem::HostIO::kChunks : 1;
    const size_t per = (P->N + io.nchunks - 1) / io.nchunks;
    for (int k = 0; k < io.nchunks; ++k) {
        const size_t o = per * k;
        if (o < P->N) {
            const size_t len = P->N - o < per ? P->N - o : per;
            cudaMemcpyAsync(u + o, u_host_in + o, len * sizeof(double), cudaMemcpyHostToDevice, io.stream);
        }
        cudaEventRecord(io.ev_chunk[k], io.stream);
    }
    cudaEventRecord(io.ev_in, io.stream);
    io.in_pending = true;
    const bool chained = !restart && P->chain_ok && P->chain_u == u;
    P->chain_ok = false;
    st = cn_drive(P, u, F_half, nullptr, u, tol, info, s, chained, nullptr, nullptr);
    io_wait_input(P, s);
    if (st == TFDE_OK && !io.out_valid) {
        // no copy was offered after the last write of u (or none at all)
        if (io.out_pending) cudaStreamWaitEvent(s, io.ev_out, 0);
        cudaMemcpyAsync(u_host_out, u, bytes, cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t e1 = cudaStreamSynchronize(io.stream);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    io.in = nullptr;
    io.out = nullptr;
    io.dev = nullptr;
    io.in_pending = io.out_pending = io.out_valid = false;
    io.nchunks = 1;
    if (st == TFDE_OK && (e1 != cudaSuccess || e2 != cudaSuccess))
        st = set_error(TFDE_ECUDA, std::string("host copies: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    if (st == TFDE_OK) {
        P->chain_ok = true;
        P->chain_u = u;
    }
    return st;
}

int tfde_cn_advance_guess(const tfde_problem* prob, double* u, const double* F_half, const double* x0, int restart,
                          double tol, tfde_info* info, int* used_guess, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_dev(x0, "x0")) || (st = check_tol(tol))) return st;
    if (F_half && (st = check_dev(F_half, "F_half"))) return st;
    if (F_half == u || x0 == u) return set_error(TFDE_EINVAL, "F_half or x0 aliases u");
    tfde_problem* P = const_cast<tfde_problem*>(prob);
    const bool chained = !restart && P->chain_ok && P->chain_u == u;
    P->chain_ok = false;
    st = cn_drive(P, u, F_half, nullptr, u, tol, info, (cudaStream_t)stream, chained, x0, used_guess);
    if (st == TFDE_OK) {
        P->chain_ok = true;
        P->chain_u = u;
    }
    return st;
}

int tfde_set_guess_order(tfde_problem* prob, int order) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    if (order < 0 || order > 3) return set_error(TFDE_EINVAL, "guess order must be 0, 1, 2 or 3");
    if (order > 0)
        if (int st = ensure_history(prob)) return st;
    prob->guess_order = order;
    return TFDE_OK;
}

int tfde_batch_create(const tfde_params* params, int count, int restart, void* stream, tfde_batch** out) {
    if (!params || !out) return set_error(TFDE_EINVAL, "NULL argument");
    *out = nullptr;
    int st = pre_call();
    if (st) return st;
    return batch_create(params, count, restart, (cudaStream_t)stream, out);
}

int tfde_batch_destroy(tfde_batch* batch) { return batch_destroy(batch); }

int tfde_batch_cn_advance(tfde_batch* batch, double* const* u, const double* const* F_half, int restart, double tol,
                          tfde_info* infos, void* stream) {
    if (!batch || !u) return set_error(TFDE_EINVAL, "NULL argument");
    int st;
    if ((st = pre_call()) || (st = check_tol(tol))) return st;
    const int C = tfde_batch_count(batch);
    for (int i = 0; i < C; ++i) {
        if ((st = check_dev(u[i], "u[i]"))) return st;
        if (F_half && F_half[i] && (st = check_dev(F_half[i], "F_half[i]"))) return st;
        if (F_half && F_half[i] == u[i]) return set_error(TFDE_EINVAL, "F_half[i] aliases u[i]");
        for (int k = 0; k < i; ++k)
            if (u[k] == u[i]) return set_error(TFDE_EINVAL, "two problems share one u buffer");
    }
    return batch_cn_advance(batch, u, F_half, restart, tol, infos, (cudaStream_t)stream);
}

int tfde_cnn_create(const int n[3], tfde_cnn** out) {
    if (!n || !out) return set_error(TFDE_EINVAL, "NULL argument");
    *out = nullptr;
    int st = pre_call();
    if (st) return st;
    return cnn::cnn_create(n, out);
}

int tfde_cnn_destroy(tfde_cnn* net) { return cnn::cnn_destroy(net); }

int tfde_cnn_set_params(tfde_cnn* net, const float* params) {
    if (!net || !params) return set_error(TFDE_EINVAL, "NULL argument");
    return cnn::cnn_set_params(net, params);
}

int tfde_cnn_get_params(const tfde_cnn* net, float* params) {
    if (!net || !params) return set_error(TFDE_EINVAL, "NULL argument");
    return cnn::cnn_get(net, 0, params);
}

int tfde_cnn_get_grads(const tfde_cnn* net, float* grads) {
    if (!net || !grads) return set_error(TFDE_EINVAL, "NULL argument");
    return cnn::cnn_get(net, 1, grads);
}

int tfde_cnn_predict(tfde_cnn* net, const double* u, const double* dtF, const double* coef, double* x0, void* stream) {
    if (!net || !coef) return set_error(TFDE_EINVAL, "NULL argument");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_dev(x0, "x0"))) return st;
    if (dtF && (st = check_dev(dtF, "dtF"))) return st;
    return cnn::cnn_predict(net, u, nullptr, nullptr, dtF, coef, x0, (cudaStream_t)stream);
}

int tfde_cnn_predict_hist(tfde_cnn* net, const double* u, const double* u1, const double* u2, const double* dtF,
                          const double* coef, double* x0, void* stream) {
    if (!net || !coef) return set_error(TFDE_EINVAL, "NULL argument");
    if (u2 && !u1) return set_error(TFDE_EINVAL, "u2 needs u1");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_dev(x0, "x0"))) return st;
    if (dtF && (st = check_dev(dtF, "dtF"))) return st;
    if (u1 && (st = check_dev(u1, "u1"))) return st;
    if (u2 && (st = check_dev(u2, "u2"))) return st;
    return cnn::cnn_predict(net, u, u1, u2, dtF, coef, x0, (cudaStream_t)stream);
}

int tfde_cnn_accumulate(tfde_cnn* net, const double* u, const double* dtF, const double* coef, const double* u_next,
                        double* loss, void* stream) {
    if (!net || !coef) return set_error(TFDE_EINVAL, "NULL argument");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_dev(u_next, "u_next"))) return st;
    if (dtF && (st = check_dev(dtF, "dtF"))) return st;
    return cnn::cnn_accumulate(net, u, nullptr, nullptr, dtF, coef, u_next, loss, (cudaStream_t)stream);
}

int tfde_cnn_accumulate_hist(tfde_cnn* net, const double* u, const double* u1, const double* u2, const double* dtF,
                             const double* coef, const double* u_next, double* loss, void* stream) {
    if (!net || !coef) return set_error(TFDE_EINVAL, "NULL argument");
    if (u2 && !u1) return set_error(TFDE_EINVAL, "u2 needs u1");
    int st;
    if ((st = pre_call()) || (st = check_dev(u, "u")) || (st = check_dev(u_next, "u_next"))) return st;
    if (dtF && (st = check_dev(dtF, "dtF"))) return st;
    if (u1 && (st = check_dev(u1, "u1"))) return st;
    if (u2 && (st = check_dev(u2, "u2"))) return st;
    return cnn::cnn_accumulate(net, u, u1, u2, dtF, coef, u_next, loss, (cudaStream_t)stream);
}

int tfde_cnn_adam_step(tfde_cnn* net, float lr, void* stream) {
    if (!net) return set_error(TFDE_EINVAL, "NULL argument");
    if (!(lr > 0.f)) return set_error(TFDE_EINVAL, "learning rate must be > 0");
    return cnn::cnn_adam(net, lr, (cudaStream_t)stream);
}

int tfde_source_example2(const tfde_problem* prob, double cP, double cS, double* F, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    int st;
    if ((st = pre_call()) || (st = check_dev(F, "F"))) return st;
    if (!prob->have_src) return set_error(TFDE_EINVAL, "Example 2 source needs Omega = (0,1)^3");
    launch_source_assemble_f64(prob->src1d, prob->n, cP, cS, F, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TFDE_OK : set_error(TFDE_ECUDA, cudaGetErrorString(e));
}

int tfde_coefficients(const tfde_problem* prob, int axis, double* q, double* lam_tau, double* eta) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    if (axis < 0 || axis > 2) return set_error(TFDE_EINVAL, "axis must be 0, 1 or 2");
    if (q)
        for (size_t k = 0; k < prob->q[axis].size(); ++k) q[k] = prob->q[axis][k];
    if (lam_tau)
        for (size_t k = 0; k < prob->lam_tau[axis].size(); ++k) lam_tau[k] = prob->lam_tau[axis][k];
    if (eta) *eta = prob->eta[axis];
    return TFDE_OK;
}

int tfde_host_coefficients(const tfde_params* params, int axis, double* q, double* lam_tau, double* lam_mass,
                           double* eta) {
    if (!params) return set_error(TFDE_EINVAL, "NULL params");
    return host_coefficients(params, axis, q, lam_tau, lam_mass, eta);
}

int tfde_stats_reset(int time_tc) { return stats_reset(time_tc); }

int tfde_stats_get(tfde_stats* out) {
    if (!out) return set_error(TFDE_EINVAL, "NULL stats");
    return stats_get(out);
}

int tfde_spectrum(const tfde_params* params, int steps, const double* v0, tfde_spectrum_info* out, void* stream) {
    if (!params || !out) return set_error(TFDE_EINVAL, "NULL params or output");
    if (steps < 2 || steps > 500) return set_error(TFDE_EINVAL, "steps must lie in 2..500");
    if (int st = check_dev(v0, "v0")) return st;
    if (int st = pre_call()) return st;
    return spectrum(params, steps, v0, out, (cudaStream_t)stream);
}

int tfde_set_device_loop(tfde_problem* prob, int enable) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    return mixed_set_device_loop(prob, enable);
}

long long tfde_device_loop_launches(const tfde_problem* prob) { return prob ? mixed_graph_launches(prob) : 0; }

int tfde_set_spectral_inner(tfde_problem* prob, int enable) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    return mixed_set_spectral(prob, enable);
}

int tfde_tune(tfde_problem* prob, int reps, void* stream) {
    if (!prob) return set_error(TFDE_EINVAL, "NULL problem");
    if (int st = pre_call()) return st;
    return mixed_tune(prob, reps, (cudaStream_t)stream);
}

int tfde_batch_tune(tfde_batch* batch, int reps, void* stream) {
    if (!batch) return set_error(TFDE_EINVAL, "NULL batch");
    if (int st = pre_call()) return st;
    return batch_tune(batch, reps, (cudaStream_t)stream);
}

int tfde_tune_get(tfde_tune_entry* out, int cap, int* count) {
    if ((!out && cap > 0) || cap < 0) return set_error(TFDE_EINVAL, "NULL output or negative capacity");
    return tc::tune_export(out, cap, count);
}

int tfde_tune_set(const tfde_tune_entry* in, int count) {
    if ((!in && count > 0) || count < 0) return set_error(TFDE_EINVAL, "NULL input or negative count");
    return tc::tune_import(in, count);
}

int tfde_tune_clear(void) {
    tc::tune_clear();
    return TFDE_OK;
}

int tfde_selftest_wait(long long limit_ns, int* tmem_freed, void* stream) {
    if (int st = pre_call()) return st;
    return tc::wait_selftest(limit_ns, tmem_freed, (cudaStream_t)stream);
}

const char* tfde_last_error(void) { return last_error_text(); }

const char* tfde_version(void) { return "tfde-gb300 0.1 (sm_103a)"; }

}  // extern "C"
