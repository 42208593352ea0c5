// Ensembles: many independent meshes of mixed degree advanced together.
//
// The instances of one degree are concatenated into one group context: their
// elements back to back, their connectivity shifted by the element offset,
// and an element -> instance map that gives every instance its own time
// step. A step of the whole ensemble is one CUDA graph in which the groups are
// parallel branches; the graph is captured once per (state pointer, dt) and
// replayed for every step, so the host issues one launch per step however
// many instances there are. Every kernel computes each element (face, node)
// exactly as for a single mesh, so an instance's result is bitwise the result
// of swe_step on that instance alone.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "swe_internal.h"

struct swe_ens {
    int device = 0;
    int ninst = 0;
    swe_params p{};
    std::vector<swe_ctx*> groups;   // one per degree, increasing N
    std::vector<int64_t> goff;      // base of every group's planes in W (doubles)
    std::vector<int> gcount;        // instances per group
    std::vector<int> ig, il;        // instance -> group, index within the group
    std::vector<int64_t> ie0;       // instance -> first element within its group
    std::vector<int> iK;            // instance -> elements
    int64_t total = 0;              // doubles of an ensemble state
    int* status = nullptr;          // device status word shared by the groups
    std::vector<long long*> ebeg;   // per group, device [count + 1] element ranges
    double* integ = nullptr;        // device [ninst][4], group order
    std::vector<double> integ_host;
    cudaStream_t cap = nullptr;     // capture origin
    std::vector<cudaStream_t> side; // one branch per group
    std::vector<cudaEvent_t> ev;    // ev[0] fork, ev[1 + g] join of group g
    cudaGraphExec_t exec = nullptr;
    const double* graph_W = nullptr;
    double graph_dt = 0.0;
    int64_t kernels_per_step = 0;
    int64_t launches = 0;
};

namespace {

constexpr int64_t kAlign = 32;  // group planes start on 256-byte boundaries

int efail(int code, const std::string& msg) { return swe::set_last_error(code, msg); }

int ecuda(cudaError_t e, const char* where) {
    return efail(SWE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void release(swe_ens* e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (cudaEvent_t v : e->ev) cudaEventDestroy(v);
    for (cudaStream_t s : e->side) cudaStreamDestroy(s);
    if (e->cap) cudaStreamDestroy(e->cap);
    for (swe_ctx* c : e->groups) swe_destroy(c);
    for (long long* p : e->ebeg) cudaFree(p);
    if (e->integ) cudaFree(e->integ);
    if (e->status) cudaFree(e->status);
    delete e;
}

int64_t group_nodes(const swe_ctx* c) { return (int64_t)c->m.KN; }

int64_t sum_launches(const swe_ens* e) {
    int64_t s = 0;
    for (const swe_ctx* c : e->groups) s += c->launches;
    return s;
}

int check_ens(const swe_ens* e, const double* W) {
    if (!e || !W) return efail(SWE_ERR_ARG, "swe_ens: NULL argument");
    return SWE_OK;
}

}  // namespace

extern "C" int swe_ens_create(int ninst, const swe_instance* in, double g, const swe_params* p, swe_ens** out) {
    if (!out) return efail(SWE_ERR_ARG, "swe_ens_create: out is NULL");
    *out = nullptr;
    if (ninst < 1 || !in || !p) return efail(SWE_ERR_ARG, "swe_ens_create: bad argument");
    std::vector<int> degrees;
    for (int i = 0; i < ninst; ++i) {
        const swe_instance& q = in[i];
        if (q.N < 1 || q.N > SWE_NMAX || q.K < 1 || !q.x || !q.y || !q.b || !q.EToE || !q.EToF || !q.flip)
            return efail(SWE_ERR_ARG, "swe_ens_create: instance " + std::to_string(i) + ": bad size or NULL input");
        for (int64_t t = 0; t < 4 * (int64_t)q.K; ++t)
            if (q.EToE[t] < -1 || q.EToE[t] >= q.K)
                return efail(SWE_ERR_ARG, "swe_ens_create: instance " + std::to_string(i) +
                                              ": EToE outside the instance (-1 marks a wall)");
        degrees.push_back(q.N);
    }
    std::sort(degrees.begin(), degrees.end());
    degrees.erase(std::unique(degrees.begin(), degrees.end()), degrees.end());

    swe_ens* e = new swe_ens();
    cudaGetDevice(&e->device);
    e->ninst = ninst;
    e->p = *p;
    e->ig.resize(ninst);
    e->il.resize(ninst);
    e->ie0.resize(ninst);
    e->iK.resize(ninst);
    cudaError_t err = cudaMalloc(&e->status, sizeof(int));
    if (err != cudaSuccess) { release(e); return ecuda(err, "swe_ens_create: allocation"); }
    cudaMemset(e->status, 0, sizeof(int));

    const int G = (int)degrees.size();
    int64_t off = 0;
    for (int gi = 0; gi < G; ++gi) {
        const int N = degrees[gi], n = N + 1, nn = n * n;
        std::vector<int> members;
        int64_t Kg = 0;
        for (int i = 0; i < ninst; ++i)
            if (in[i].N == N) {
                e->ig[i] = gi;
                e->il[i] = (int)members.size();
                e->ie0[i] = Kg;
                e->iK[i] = in[i].K;
                members.push_back(i);
                Kg += in[i].K;
            }
        if (Kg > 0x7fffffff / nn) {
            release(e);
            return efail(SWE_ERR_ARG, "swe_ens_create: too many nodes of degree " + std::to_string(N));
        }
        std::vector<double> x(Kg * nn), y(Kg * nn), b(Kg * nn);
        std::vector<int32_t> E2E(4 * Kg), E2F(4 * Kg), fl(4 * Kg), inst(Kg);
        std::vector<long long> eb(members.size() + 1, 0);
        for (size_t mi = 0; mi < members.size(); ++mi) {
            const swe_instance& q = in[members[mi]];
            const int64_t e0 = e->ie0[members[mi]];
            memcpy(&x[e0 * nn], q.x, sizeof(double) * q.K * nn);
            memcpy(&y[e0 * nn], q.y, sizeof(double) * q.K * nn);
            memcpy(&b[e0 * nn], q.b, sizeof(double) * q.K * nn);
            for (int64_t t = 0; t < 4 * (int64_t)q.K; ++t) {
                E2E[4 * e0 + t] = q.EToE[t] < 0 ? -1 : (int32_t)(q.EToE[t] + e0);
                E2F[4 * e0 + t] = q.EToF[t];
                fl[4 * e0 + t] = q.flip[t];
            }
            for (int k = 0; k < q.K; ++k) inst[e0 + k] = (int32_t)mi;
            eb[mi + 1] = eb[mi] + q.K;
        }
        swe_ctx* c = nullptr;
        int rc = swe::create_ctx(N, (int)Kg, x.data(), y.data(), E2E.data(), E2F.data(), fl.data(), b.data(), g, p,
                                 inst.data(), (int)members.size(), e->status, &c);
        if (rc) {
            std::string msg = swe_last_error();
            release(e);
            return efail(rc, "swe_ens_create: degree " + std::to_string(N) + ": " + msg);
        }
        e->groups.push_back(c);
        e->gcount.push_back((int)members.size());
        e->goff.push_back(off);
        off += (3 * Kg * nn + kAlign - 1) / kAlign * kAlign;
        long long* d = nullptr;
        err = cudaMalloc(&d, sizeof(long long) * eb.size());
        if (err == cudaSuccess) {
            e->ebeg.push_back(d);
            err = cudaMemcpy(d, eb.data(), sizeof(long long) * eb.size(), cudaMemcpyHostToDevice);
        }
        if (err != cudaSuccess) { release(e); return ecuda(err, "swe_ens_create: upload"); }
    }
    e->total = off;
    e->integ_host.resize(4 * (size_t)ninst);
    err = cudaMalloc(&e->integ, sizeof(double) * 4 * ninst);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
    for (int gi = 0; gi < G && err == cudaSuccess; ++gi) {
        cudaStream_t s = nullptr;
        err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (err == cudaSuccess) e->side.push_back(s);
    }
    for (int v = 0; v < G + 1 && err == cudaSuccess; ++v) {
        cudaEvent_t ev = nullptr;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err == cudaSuccess) e->ev.push_back(ev);
    }
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) { release(e); return ecuda(err, "swe_ens_create"); }
    *out = e;
    return SWE_OK;
}

extern "C" void swe_ens_destroy(swe_ens* e) {
    if (!e) return;
    cudaDeviceSynchronize();
    release(e);
}

extern "C" int swe_ens_size(const swe_ens* e, int64_t* total, int* ngroups) {
    if (!e) return efail(SWE_ERR_ARG, "swe_ens_size: NULL ensemble");
    if (total) *total = e->total;
    if (ngroups) *ngroups = (int)e->groups.size();
    return SWE_OK;
}

extern "C" int swe_ens_layout(const swe_ens* e, int i, int64_t* offset, int64_t* plane_stride, int* N, int* K) {
    if (!e) return efail(SWE_ERR_ARG, "swe_ens_layout: NULL ensemble");
    if (i < 0 || i >= e->ninst) return efail(SWE_ERR_ARG, "swe_ens_layout: instance out of range");
    const swe_ctx* c = e->groups[e->ig[i]];
    const int64_t nn = (int64_t)c->m.n * c->m.n;
    if (offset) *offset = e->goff[e->ig[i]] + e->ie0[i] * nn;
    if (plane_stride) *plane_stride = group_nodes(c);
    if (N) *N = c->m.N;
    if (K) *K = e->iK[i];
    return SWE_OK;
}

extern "C" int swe_ens_rhs(swe_ens* e, const double* W, double* R, void* stream) {
    if (int rc = check_ens(e, W)) return rc;
    if (!R || W == R) return efail(SWE_ERR_ARG, "swe_ens_rhs: R is NULL or equal to W");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t before = sum_launches(e);
    for (size_t gi = 0; gi < e->groups.size(); ++gi)
        swe::rhs_chain(e->groups[gi], W + e->goff[gi], R + e->goff[gi], s, nullptr, false);
    e->launches += sum_launches(e) - before;
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SWE_OK : ecuda(err, "swe_ens_rhs");
}

extern "C" int swe_ens_max_dt(swe_ens* e, const double* W, double* dt_cfl, double* dt_pos, void* stream) {
    if (int rc = check_ens(e, W)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t before = sum_launches(e);
    std::vector<double> host;
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
        swe_ctx* c = e->groups[gi];
        swe::launch_prim(c, W + e->goff[gi], s, nullptr);
        if (c->kv > 0.0) swe::launch_indicator(c, W + e->goff[gi], s, nullptr);  // viscosities (viscous restriction)
        swe::launch_dt(c, W + e->goff[gi], 0.0, s, nullptr);
    }
    e->launches += sum_launches(e) - before;
    std::vector<std::vector<double>> per(e->groups.size());
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
        per[gi].resize(3 * (size_t)e->gcount[gi]);
        cudaMemcpyAsync(per[gi].data(), e->groups[gi]->w.dt, sizeof(double) * per[gi].size(), cudaMemcpyDeviceToHost,
                        s);
    }
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return ecuda(err, "swe_ens_max_dt");
    for (int i = 0; i < e->ninst; ++i) {
        const int gi = e->ig[i], cnt = e->gcount[gi];
        if (dt_cfl) dt_cfl[i] = per[gi][cnt + e->il[i]];
        if (dt_pos) dt_pos[i] = per[gi][2 * cnt + e->il[i]];
    }
    err = cudaGetLastError();
    return err == cudaSuccess ? SWE_OK : ecuda(err, "swe_ens_max_dt");
}

namespace {

// Capture one step of every group as parallel branches of a graph.
int capture_step(swe_ens* e, double* W, double dt) {
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    const int64_t before = sum_launches(e);
    cudaError_t err = cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return ecuda(err, "swe_ens_step: begin capture");
    // The start states are saved before the branches fork: a failure in one
    // branch stops every later kernel, and must not stop another group's copy.
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
        swe_ctx* c = e->groups[gi];
        swe::launch_copy(c, W + e->goff[gi], c->w.Wn, 3 * c->m.KN, e->cap, e->status);
    }
    cudaEventRecord(e->ev[0], e->cap);
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
        cudaStreamWaitEvent(e->side[gi], e->ev[0], 0);
        swe::step_once(e->groups[gi], W + e->goff[gi], dt, e->side[gi], e->status, false);
        cudaEventRecord(e->ev[1 + gi], e->side[gi]);
        cudaStreamWaitEvent(e->cap, e->ev[1 + gi], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t end = cudaStreamEndCapture(e->cap, &graph);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (end != cudaSuccess || err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return ecuda(end != cudaSuccess ? end : err, "swe_ens_step: capture");
    }
    err = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        e->exec = nullptr;
        return ecuda(err, "swe_ens_step: instantiate");
    }
    e->graph_W = W;
    e->graph_dt = dt;
    e->kernels_per_step = sum_launches(e) - before;
    return SWE_OK;
}

}  // namespace

extern "C" int swe_ens_step(swe_ens* e, double* W, double dt, int nsteps, double* dt_last, void* stream) {
    if (int rc = check_ens(e, W)) return rc;
    if (nsteps < 0) return efail(SWE_ERR_ARG, "swe_ens_step: nsteps < 0");
    const bool adaptive = !(dt > 0.0);
    if (adaptive && !(e->p.cfl > 0.0)) return efail(SWE_ERR_ARG, "swe_ens_step: dt <= 0 needs cfl > 0");
    if (adaptive) dt = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps == 0) return SWE_OK;
    // Capturing only records the launches; nothing runs until the replays.
    if (!e->exec || e->graph_W != W || e->graph_dt != dt)
        if (int rc = capture_step(e, W, dt)) return rc;
    cudaMemsetAsync(e->status, 0, sizeof(int), s);
    const int64_t before = sum_launches(e);
    // Velocities of the start state; every later stage update writes them.
    for (size_t gi = 0; gi < e->groups.size(); ++gi)
        swe::launch_prim(e->groups[gi], W + e->goff[gi], s, e->status);
    e->launches += sum_launches(e) - before;
    for (int st = 0; st < nsteps; ++st) {
        cudaError_t err = cudaGraphLaunch(e->exec, s);
        if (err != cudaSuccess) return ecuda(err, "swe_ens_step: graph launch");
    }
    e->launches += e->kernels_per_step * nsteps;
    int status = 0;
    cudaMemcpyAsync(&status, e->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    std::vector<std::vector<double>> dts(e->groups.size());
    if (adaptive && dt_last)
        for (size_t gi = 0; gi < e->groups.size(); ++gi) {
            dts[gi].resize(e->gcount[gi]);
            cudaMemcpyAsync(dts[gi].data(), e->groups[gi]->w.dt, sizeof(double) * e->gcount[gi],
                            cudaMemcpyDeviceToHost, s);
        }
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return ecuda(err, "swe_ens_step");
    if (dt_last)
        for (int i = 0; i < e->ninst; ++i) dt_last[i] = adaptive ? dts[e->ig[i]][e->il[i]] : dt;
    if (status) {
        cudaMemsetAsync(e->status, 0, sizeof(int), s);
        for (size_t gi = 0; gi < e->groups.size(); ++gi)
            cudaMemcpyAsync(W + e->goff[gi], e->groups[gi]->w.Wn, sizeof(double) * 3 * group_nodes(e->groups[gi]),
                            cudaMemcpyDeviceToDevice, s);
        err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return ecuda(err, "swe_ens_step: rollback");
        if (status & 2)
            return efail(SWE_ERR_NONFINITE, "swe_ens_step: non-finite state; rolled back the failing step");
        return efail(SWE_ERR_NEG_MEAN,
                     "swe_ens_step: negative element mean water height; rolled back the failing step");
    }
    err = cudaGetLastError();
    return err == cudaSuccess ? SWE_OK : ecuda(err, "swe_ens_step");
}

extern "C" int swe_ens_integrals(swe_ens* e, const double* W, double* out, void* stream) {
    if (int rc = check_ens(e, W)) return rc;
    if (!out) return efail(SWE_ERR_ARG, "swe_ens_integrals: out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t before = sum_launches(e);
    int64_t base = 0;
    for (size_t gi = 0; gi < e->groups.size(); ++gi) {
        swe::launch_prim(e->groups[gi], W + e->goff[gi], s, nullptr);  // velocities for the kinetic energy
        swe::launch_reduce_inst(e->groups[gi], W + e->goff[gi], e->ebeg[gi], e->integ + 4 * base, s);
        base += e->gcount[gi];
    }
    e->launches += sum_launches(e) - before;
    cudaMemcpyAsync(e->integ_host.data(), e->integ, sizeof(double) * 4 * e->ninst, cudaMemcpyDeviceToHost, s);
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return ecuda(err, "swe_ens_integrals");
    std::vector<int64_t> gbase(e->groups.size(), 0);
    for (size_t gi = 1; gi < e->groups.size(); ++gi) gbase[gi] = gbase[gi - 1] + e->gcount[gi - 1];
    for (int i = 0; i < e->ninst; ++i)
        for (int c = 0; c < 4; ++c) out[4 * i + c] = e->integ_host[4 * (gbase[e->ig[i]] + e->il[i]) + c];
    err = cudaGetLastError();
    return err == cudaSuccess ? SWE_OK : ecuda(err, "swe_ens_integrals");
}

extern "C" int64_t swe_ens_launches(const swe_ens* e) { return e ? e->launches : 0; }

extern "C" int swe_ens_autotune(swe_ens* e, const double* W, void* stream) {
    if (int rc = check_ens(e, W)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t before = sum_launches(e);
    for (size_t gi = 0; gi < e->groups.size(); ++gi)
        if (int rc = swe::autotune_ctx(e->groups[gi], W + e->goff[gi], s)) return rc;
    e->launches += sum_launches(e) - before;
    // The captured step holds the old shapes: capture again at the next step.
    if (e->exec) {
        cudaError_t err = cudaDeviceSynchronize();
        if (err != cudaSuccess) return ecuda(err, "swe_ens_autotune");
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    return SWE_OK;
}

extern "C" int swe_ens_group(const swe_ens* e, int group, int* N, int* members, int* vol_threads,
                             int* upd_warps) {
    if (!e) return efail(SWE_ERR_ARG, "swe_ens_group: NULL ensemble");
    if (group < 0 || group >= (int)e->groups.size()) return efail(SWE_ERR_ARG, "swe_ens_group: group out of range");
    const swe_ctx* c = e->groups[group];
    if (N) *N = c->m.N;
    if (members) *members = e->gcount[group];
    if (vol_threads) *vol_threads = c->vol_tpb;
    if (upd_warps) *upd_warps = c->upd_wpb;
    return SWE_OK;
}
