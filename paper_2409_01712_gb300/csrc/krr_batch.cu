// Batched KRR: many (cohort, fold, lambda) problems of uneven size -- the
// paper picks gamma and alpha by cross-validation (Sec. III), which means
// solving many such problems.  Every problem gets its own context and
// stream; the whole set (Build, Factor, Solve, Predict of every problem) is
// captured once into one CUDA graph with a fork/join over the problem
// streams, so independent problems overlap on the GPU and a run is a single
// graph launch.  An autotuner picks the tile edge per problem size from
// timed trial runs.  Problems that differ only in lambda (the same genotype
// matrix, gamma and tile) share one Build: the first of them builds the
// kernel matrix, the others wait for it on their streams and factorise the
// same tiles (K does not depend on lambda; nothing after the Build writes it).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "krr_internal.h"

struct krr_batch {
    krr_options opt;
    cudaStream_t main = nullptr;     // caller's stream: trials and graph launches
    cudaStream_t capture = nullptr;  // own stream the graph is captured on (the
                                     // caller's may be the legacy default stream,
                                     // which cannot be captured)
    int64_t m = 0, p = 0;
    std::vector<krr_batch_problem> probs;
    std::vector<krr_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<int32_t> tiles;
    std::vector<int32_t> owner;       // problem whose Build this one reads (itself when it builds)
    std::vector<cudaEvent_t> built;   // recorded after an owner's Build
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double> tune_ms;      // autotune level 2: ms per run of each candidate assignment
    std::string last_error;
};

namespace {

thread_local std::string g_batch_create_error;

// CTAs per launch of a batched problem: the problems run concurrently on their
// streams, and persistent kernels sized for the whole GPU would each hold every
// SM while waiting on their dependency chains.  Measured on the
// cross-validation workload (64 problems, N up to 16384): no cap 408 ms per
// run; 32 CTAs for every kernel 220 ms; per class as below 183-185 ms (the
// diagonal step, mostly waiting CTAs, at 12; the sweeps at 16; the tensor-core
// kernels, which keep their CTAs busy, at 64).  Later re-measured around
// these caps (172-176 ms): the diagonal step at 4 / 6 CTAs 204 / 185 ms,
// at 16 / 24 (with the lookahead) 175 / 187 ms; diagonal step and sweeps
// both at 8 195 ms; the pair kernels at 48 (sweeps 12) 194 ms: the chain of
// the diagonal steps of the largest problems needs their CTAs, and more
// CTAs crowd out the other problems.
constexpr int BATCH_CTA_CAP = 32;
constexpr int BATCH_CAP_DIAG = 12, BATCH_CAP_SWEEP = 16, BATCH_CAP_PAIR = 64, BATCH_CAP_SINGLE = 64;

void set_batch_caps(krr_ctx *c) {
    krr::Ctx *cc = reinterpret_cast<krr::Ctx *>(c);
    cc->cta_cap = BATCH_CTA_CAP;
    cc->cta_caps[krr::GL_DIAG] = BATCH_CAP_DIAG;
    cc->cta_caps[krr::GL_SWEEP] = BATCH_CAP_SWEEP;
    cc->cta_caps[krr::GL_PAIR] = BATCH_CAP_PAIR;
    cc->cta_caps[krr::GL_SINGLE] = BATCH_CAP_SINGLE;
}

// Build (or, with src != NULL, wait for src's Build and read it), Factor,
// Solve and Predict of one problem on c's stream; `done` is recorded after
// an own Build.
krr_status issue(krr_ctx *c, const krr_batch_problem &pr, int64_t m, int64_t p, krr_ctx *src = nullptr,
                 cudaEvent_t src_built = nullptr, cudaEvent_t done = nullptr) {
    krr::Ctx *cc = reinterpret_cast<krr::Ctx *>(c);
    if (src) {
        if (cudaStreamWaitEvent(cc->stream, src_built, 0) != cudaSuccess) return KRR_ECUDA;
        KRR_TRY(krr::adopt_build(cc, reinterpret_cast<krr::Ctx *>(src)));
    } else {
        KRR_TRY(krr_build_kernel(c, pr.G, pr.n, m, pr.ldg, pr.gamma));
        if (done && cudaEventRecord(done, cc->stream) != cudaSuccess) return KRR_ECUDA;
    }
    KRR_TRY(krr_factor(c, pr.lambda, nullptr));
    krr_status st = krr_solve(c, pr.Y, p, pr.ldy, pr.A, pr.lda, nullptr);
    if (st != KRR_OK) return st;
    if (pr.T && pr.n_test > 0) KRR_TRY(krr_predict(c, pr.T, pr.n_test, pr.ldt, pr.A, pr.lda, p, pr.Yt, pr.ldyt));
    return KRR_OK;
}

// Wall time (ms) of one eager pipeline of problem pr with tile b.
krr_status trial_ms(const krr_options &base, cudaStream_t s, const krr_batch_problem &pr, int64_t m, int64_t p,
                    int64_t b, double *ms, std::string *why) {
    krr_options o = base;
    o.tile = b;
    krr_ctx *c = nullptr;
    KRR_TRY(krr_create(&c, &o, s));
    reinterpret_cast<krr::Ctx *>(c)->graph_mode = 1;
    set_batch_caps(c);
    if (krr::ensure_lookahead_stream(reinterpret_cast<krr::Ctx *>(c)) != KRR_OK) {
        krr_destroy(c);
        return KRR_ECUDA;
    }
    krr_status st = issue(c, pr, m, p);  // warm-up (allocations)
    if (st == KRR_OK) {
        cudaStreamSynchronize(s);
        const auto t0 = std::chrono::steady_clock::now();
        st = issue(c, pr, m, p);
        cudaStreamSynchronize(s);
        *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (st != KRR_OK && why) *why = krr_last_error(c);
    krr_destroy(c);
    return st;
}

// Contexts, streams and the captured graph of the current tile assignment
// bt->tiles: problems sharing a Build (same genotypes, shape, gamma and
// tile) are found, every pipeline runs once eagerly (allocations), then all
// are captured into one graph with a fork / join over the problem streams.
krr_status instantiate(krr_batch *bt, std::string *msg) {
    const int32_t count = (int32_t)bt->probs.size();
    const krr_batch_problem *problems = bt->probs.data();
    const int64_t m = bt->m, p = bt->p;
    // problems are captured by decreasing N (stable: the first problem of a
    // shared Build stays ahead of the others), so the longest dependency
    // chains start first: 168-169 ms per run on the cross-validation
    // workload against 168-173 ms in problem order (stream priorities by
    // size on top of it changed nothing)
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b2) { return problems[a].n > problems[b2].n; });
    bt->owner.assign(count, -1);
    for (int32_t i = 0; i < count; ++i) {
        bt->owner[i] = i;
        for (int32_t j = 0; j < i; ++j) {
            const krr_batch_problem &a = problems[i], &b2 = problems[j];
            if (bt->owner[j] == j && a.G == b2.G && a.n == b2.n && a.ldg == b2.ldg && a.gamma == b2.gamma &&
                bt->tiles[i] == bt->tiles[j]) {
                bt->owner[i] = j;
                break;
            }
        }
    }
    bt->ctx.assign(count, nullptr);
    bt->streams.assign(count, nullptr);
    bt->join.assign(count, nullptr);
    bt->built.assign(count, nullptr);
    for (int32_t i = 0; i < count; ++i) {
        if (cudaStreamCreateWithFlags(&bt->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&bt->join[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&bt->built[i], cudaEventDisableTiming) != cudaSuccess) {
            *msg = "stream creation failed";
            return KRR_ECUDA;
        }
        krr_options o = bt->opt;
        o.tile = bt->tiles[i];
        krr_status st = krr_create(&bt->ctx[i], &o, bt->streams[i]);
        if (st != KRR_OK) {
            *msg = std::string("krr_batch_create: ") + krr_last_error(nullptr);
            return st;
        }
        reinterpret_cast<krr::Ctx *>(bt->ctx[i])->graph_mode = 1;
        set_batch_caps(bt->ctx[i]);
        st = krr::ensure_lookahead_stream(reinterpret_cast<krr::Ctx *>(bt->ctx[i]));
        if (st != KRR_OK) {
            *msg = "krr_batch_create: lookahead stream";
            return st;
        }
        const int32_t ow = bt->owner[i];
        st = (ow == i) ? issue(bt->ctx[i], problems[i], m, p, nullptr, nullptr, bt->built[i])
                       : issue(bt->ctx[i], problems[i], m, p, bt->ctx[ow], bt->built[ow]);
        if (st != KRR_OK) {
            *msg = std::string("krr_batch_create: warm-up of problem ") + std::to_string(i) + ": " +
                   krr_last_error(bt->ctx[i]);
            return st;
        }
    }
    {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            *msg = std::string("warm-up failed: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
    }
    {
        const cudaError_t e = cudaStreamBeginCapture(bt->capture, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            *msg = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
    }
    cudaEventRecord(bt->fork, bt->capture);
    krr_status cst = KRR_OK;
    std::string cmsg;
    for (int32_t r = 0; r < count && cst == KRR_OK; ++r) {
        const int32_t i = order[r];
        cudaStreamWaitEvent(bt->streams[i], bt->fork, 0);
        const int32_t o = bt->owner[i];
        cst = (o == i) ? issue(bt->ctx[i], problems[i], m, p, nullptr, nullptr, bt->built[i])
                       : issue(bt->ctx[i], problems[i], m, p, bt->ctx[o], bt->built[o]);
        if (cst != KRR_OK) cmsg = "problem " + std::to_string(i) + ": " + krr_last_error(bt->ctx[i]);
        cudaEventRecord(bt->join[i], bt->streams[i]);
        cudaStreamWaitEvent(bt->capture, bt->join[i], 0);
    }
    const cudaError_t ce = cudaStreamEndCapture(bt->capture, &bt->graph);
    if (cst != KRR_OK || ce != cudaSuccess || !bt->graph) {
        cudaGetLastError();
        *msg = "graph capture failed: " + (cst != KRR_OK ? cmsg : std::string(cudaGetErrorString(ce)));
        return cst != KRR_OK ? cst : KRR_ECUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *msg = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

// Frees what instantiate() made; the batch can be instantiated again.
void release(krr_batch *bt) {
    if (bt->exec) cudaStreamSynchronize(bt->main);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    bt->exec = nullptr;
    bt->graph = nullptr;
    // contexts that read another's Build go first
    for (size_t i = 0; i < bt->ctx.size(); ++i)
        if (i < bt->owner.size() && bt->owner[i] != (int32_t)i) krr_destroy(bt->ctx[i]);
    for (size_t i = 0; i < bt->ctx.size(); ++i)
        if (i >= bt->owner.size() || bt->owner[i] == (int32_t)i) krr_destroy(bt->ctx[i]);
    for (cudaEvent_t e : bt->built)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : bt->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : bt->join)
        if (e) cudaEventDestroy(e);
    bt->ctx.clear();
    bt->owner.clear();
    bt->built.clear();
    bt->streams.clear();
    bt->join.clear();
}

// Median wall time of `runs` graph launches after one more (untimed); any
// per-problem error is returned.
krr_status time_graph(krr_batch *bt, int runs, double *ms) {
    std::vector<double> t;
    for (int r = 0; r <= runs; ++r) {
        const auto t0 = std::chrono::steady_clock::now();
        if (cudaGraphLaunch(bt->exec, bt->main) != cudaSuccess || cudaStreamSynchronize(bt->main) != cudaSuccess) {
            cudaGetLastError();
            return KRR_ECUDA;
        }
        if (r > 0) t.push_back(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    }
    for (krr_ctx *c : bt->ctx) {
        krr::DevErrors e;
        if (cudaMemcpy(&e, reinterpret_cast<krr::Ctx *>(c)->derr, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess)
            return KRR_ECUDA;
        if (e.code) return (krr_status)e.code;
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return KRR_OK;
}

}  // namespace

extern "C" krr_status krr_batch_create(krr_batch **out, const krr_options *opt, void *stream, int64_t m,
                                       int64_t p, const krr_batch_problem *problems, int32_t count,
                                       int32_t autotune) {
    if (!out || !problems || count < 1 || m < 1 || p < 1) return KRR_EINVAL;
    *out = nullptr;
    krr_batch *bt = new (std::nothrow) krr_batch();
    if (!bt) return KRR_ENOMEM;
    krr_default_options(&bt->opt);
    if (opt) bt->opt = *opt;
    bt->main = (cudaStream_t)stream;
    bt->m = m;
    bt->p = p;
    bt->probs.assign(problems, problems + count);
    g_batch_create_error.clear();
    auto fail = [&](krr_status st, const std::string &msg) {
        g_batch_create_error = msg;
        krr_batch_destroy(bt);
        return st;
    };
    for (int32_t i = 0; i < count; ++i) {
        const krr_batch_problem &pr = problems[i];
        if (!pr.G || !pr.Y || !pr.A || pr.n < 1 || pr.ldg < m || pr.ldy < p || pr.lda < p)
            return fail(KRR_EINVAL, "krr_batch_create: bad problem " + std::to_string(i));
    }
    // ---- autotune the tile edge: time the smallest, median and largest
    // problems with every candidate; each problem takes the candidate that was
    // fastest on the measured problem nearest to it in log N.
    bt->tiles.assign(count, (int32_t)bt->opt.tile);
    if (autotune) {
        std::vector<int32_t> order(count);
        for (int32_t i = 0; i < count; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b2) { return problems[a].n < problems[b2].n; });
        const int32_t probes[3] = {order[0], order[count / 2], order[count - 1]};
        const int64_t cand[3] = {256, 512, 1024};
        int64_t best_b[3];
        for (int q = 0; q < 3; ++q) {
            double best = INFINITY;
            best_b[q] = bt->opt.tile;
            for (int64_t b : cand) {
                if (b > 2 * ((problems[probes[q]].n + 255) / 256 * 256) && b != 256) continue;
                double ms = 0.0;
                std::string why;
                krr_status st = trial_ms(bt->opt, bt->main, problems[probes[q]], m, p, b, &ms, &why);
                if (st != KRR_OK)
                    return fail(st, "krr_batch_create: autotune trial (tile " + std::to_string(b) + ") failed: " + why);
                if (ms < best) {
                    best = ms;
                    best_b[q] = b;
                }
            }
        }
        for (int32_t i = 0; i < count; ++i) {
            int qbest = 0;
            double dist = INFINITY;
            for (int q = 0; q < 3; ++q) {
                const double d = fabs(log((double)problems[i].n) - log((double)problems[probes[q]].n));
                if (d < dist) {
                    dist = d;
                    qbest = q;
                }
            }
            bt->tiles[i] = (int32_t)best_b[qbest];
        }
    }
    if (cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&bt->capture, cudaStreamNonBlocking) != cudaSuccess)
        return fail(KRR_ECUDA, "event / stream creation failed");
    // ---- autotune level 2: the whole batch, captured and timed, with the
    // per-size choice above and with every uniform tile edge; the fastest
    // assignment is kept (the per-size trials time one problem alone, while
    // the batch runs them all at once, sharing the SMs)
    if (autotune >= 2) {
        std::vector<std::vector<int32_t>> cands;
        cands.push_back(bt->tiles);
        int64_t nmax = 0;
        for (int32_t i = 0; i < count; ++i) nmax = std::max<int64_t>(nmax, problems[i].n);
        for (int32_t b : {256, 512, 1024}) {
            if (b > 2 * nmax && b != 256) continue;
            std::vector<int32_t> u(count, b);
            if (std::find(cands.begin(), cands.end(), u) == cands.end()) cands.push_back(u);
        }
        double best = INFINITY;
        size_t best_c = 0;
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            bt->tiles = cands[ci];
            std::string msg;
            krr_status st = instantiate(bt, &msg);
            double ms = INFINITY;
            if (st == KRR_OK) st = time_graph(bt, 3, &ms);
            release(bt);
            if (st != KRR_OK) return fail(st, "krr_batch_create: autotune of the batch: " + msg);
            bt->tune_ms.push_back(ms);
            if (ms < best) {
                best = ms;
                best_c = ci;
            }
        }
        bt->tiles = cands[best_c];
    }
    {
        std::string msg;
        const krr_status st = instantiate(bt, &msg);
        if (st != KRR_OK) return fail(st, msg);
    }
    *out = bt;
    return KRR_OK;
}

extern "C" krr_status krr_batch_run(krr_batch *bt, krr_batch_result *results) {
    if (!bt || !bt->exec) return KRR_EINVAL;
    if (cudaGraphLaunch(bt->exec, bt->main) != cudaSuccess ||
        cudaStreamSynchronize(bt->main) != cudaSuccess) {
        cudaGetLastError();
        bt->last_error = "graph launch failed";
        return KRR_ECUDA;
    }
    krr_status worst = KRR_OK;
    for (size_t i = 0; i < bt->ctx.size(); ++i) {
        krr::Ctx *c = reinterpret_cast<krr::Ctx *>(bt->ctx[i]);
        krr::DevErrors e;
        double rn[2] = {0.0, 0.0};
        if (cudaMemcpy(&e, c->derr, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(rn, c->red + krr::RED_RNORM, sizeof(rn), cudaMemcpyDeviceToHost) != cudaSuccess) {
            bt->last_error = "result readback failed";
            return KRR_ECUDA;
        }
        const krr_status st = e.code ? (krr_status)e.code : KRR_OK;
        if (st != KRR_OK && worst == KRR_OK) {
            worst = st;
            bt->last_error = "problem " + std::to_string(i) + " failed with status " + std::to_string(e.code);
        }
        if (results) {
            results[i].status = st;
            results[i].tile = bt->tiles[i];
            results[i].rel_residual = rn[1] > 0 ? sqrt(rn[0] / rn[1]) : sqrt(rn[0]);
        }
    }
    return worst;
}

extern "C" const char *krr_batch_last_error(const krr_batch *bt) {
    return bt ? bt->last_error.c_str() : g_batch_create_error.c_str();
}

extern "C" void krr_batch_destroy(krr_batch *bt) {
    if (!bt) return;
    release(bt);
    if (bt->capture) cudaStreamDestroy(bt->capture);
    if (bt->fork) cudaEventDestroy(bt->fork);
    delete bt;
}
