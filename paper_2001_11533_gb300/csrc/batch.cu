// batch.cu -- native batch runtime: many independent control problems, each
// with several desired states, solved concurrently.
//
// Every (problem, desired state) pair is an independent outer CG.  The batch
// gives each problem up to `workers` solve slots: slot 0 is the problem
// itself, the others are handles from amgh_problem_share (same matrices and
// hierarchies, own work space and graphs).  Each slot has its own
// non-blocking stream and host thread and takes the columns c = s, s + w,
// ... of its problem, so the small, latency-bound coarse-level work of many
// solves overlaps on the GPU.  In block mode a slot instead takes a
// contiguous share of its problem's columns and solves them with
// amgh_solve_block (every operator applied to up to 8 columns per pass).  Host threads wait on blocking-sync events, so
// more threads than cores do not spin against each other.
#include <string.h>

#include <chrono>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

struct BatchSlot {
    amgh_problem *h = nullptr; // the problem (slot 0) or a shared handle
    cudaStream_t stream = 0;
    bool owned = false; // shared handle made by the batch
};

struct amgh_batch {
    std::vector<amgh_problem *> probs;
    std::vector<void *> old_streams;
    std::vector<std::vector<BatchSlot>> slots; // [problem][slot]
    int workers = 0;                           // slots per problem (0 = one per column)
    int block = 0;                             // 1: slots run amgh_solve_block
    int device = 0;
};

static void slot_release(BatchSlot &s)
{
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.owned) amgh_problem_destroy(s.h);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = BatchSlot();
}

static int make_slot(amgh_problem *p, bool share, BatchSlot &out)
{
    BatchSlot s;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return AMGH_ERR_CUDA;
    if (share) {
        int st = amgh_problem_share(p, &s.h);
        if (st) {
            cudaStreamDestroy(s.stream);
            return st;
        }
        s.owned = true;
    } else {
        s.h = p;
    }
    amgh_set_stream(s.h, s.stream);
    if (!s.h->wait_ev && cudaEventCreateWithFlags(&s.h->wait_ev, cudaEventBlockingSync | cudaEventDisableTiming) !=
                             cudaSuccess) {
        slot_release(s);
        return AMGH_ERR_CUDA;
    }
    out = s;
    return AMGH_OK;
}

// run fn(i) for i in [0, count) on count threads (device made current there)
template <typename F>
static void run_all(amgh_batch *b, int count, F fn)
{
    std::vector<std::thread> th;
    th.reserve(count);
    for (int i = 0; i < count; i++)
        th.emplace_back([b, i, &fn] {
            cudaSetDevice(b->device);
            fn(i);
        });
    for (auto &t : th) t.join();
}

extern "C" int amgh_batch_create(amgh_problem *const *probs, int nprob, amgh_batch **out)
{
    if (!out || !probs || nprob <= 0) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < nprob; i++)
        if (!probs[i] || probs[i]->parent) return AMGH_ERR_INVALID_ARG;
    amgh_batch *b = new (std::nothrow) amgh_batch();
    if (!b) return AMGH_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return AMGH_ERR_CUDA;
    }
    b->slots.resize(nprob);
    for (int i = 0; i < nprob; i++) {
        b->probs.push_back(probs[i]);
        b->old_streams.push_back((void *)probs[i]->stream);
        // work already queued on the caller's stream must finish first
        cudaStreamSynchronize(probs[i]->stream);
        BatchSlot s;
        int st = make_slot(probs[i], false, s);
        if (st) {
            amgh_batch_destroy(b);
            return st;
        }
        b->slots[i].push_back(s);
    }
    *out = b;
    return AMGH_OK;
}

extern "C" int amgh_batch_set_workers(amgh_batch *b, int workers)
{
    if (!b || workers < 0) return AMGH_ERR_INVALID_ARG;
    b->workers = workers;
    return AMGH_OK;
}

extern "C" int amgh_batch_set_block(amgh_batch *b, int block)
{
    if (!b || (block != 0 && block != 1)) return AMGH_ERR_INVALID_ARG;
    b->block = block;
    return AMGH_OK;
}

extern "C" int amgh_batch_setup(amgh_batch *b, const amgh_amg_opts *amg)
{
    if (!b) return AMGH_ERR_INVALID_ARG;
    int np = (int)b->probs.size();
    // shared handles hold the old hierarchy: drop them before a new setup
    for (int i = 0; i < np; i++) {
        auto &v = b->slots[i];
        while (!b->probs[i]->setup_done && v.size() > 1) {
            slot_release(v.back());
            v.pop_back();
        }
    }
    std::vector<int> st(np, AMGH_OK);
    // the batch runs its handles beside each other: no cooperative launches
    // (grid-fused V-cycle, persistent mass CG), which would compete for
    // residency with the other handles' kernels
    amgh_amg_opts o;
    if (amg) o = *amg;
    else amgh_amg_opts_default(&o);
    if (o.fuse_coarse == 2) o.fuse_coarse = 0;
    o.persistent_cg = 0;
    for (int i = 0; i < np; i++) b->probs[i]->in_batch = 1;
    run_all(b, np, [&](int i) {
        if (!b->probs[i]->setup_done) st[i] = amgh_amg_setup(b->probs[i], &o);
    });
    for (int s : st)
        if (s != AMGH_OK) return s;
    return AMGH_OK;
}

extern "C" int amgh_batch_solve(amgh_batch *b, const double *const *yd, const int *ncols, double *const *u,
                                const amgh_solve_opts *opts, amgh_solve_info *info)
{
    if (!b || !yd || !ncols || !u) return AMGH_ERR_INVALID_ARG;
    int np = (int)b->probs.size();
    for (int i = 0; i < np; i++)
        if (ncols[i] < 0 || (ncols[i] > 0 && (!yd[i] || !u[i]))) return AMGH_ERR_INVALID_ARG;
    // hierarchies first (concurrently), then the slots each problem needs
    std::vector<int> pst(np, AMGH_OK);
    run_all(b, np, [&](int i) {
        if (!b->probs[i]->setup_done) pst[i] = amgh_amg_setup(b->probs[i], nullptr);
    });
    struct Work {
        int prob, slot, nslot;
    };
    std::vector<Work> work;
    for (int i = 0; i < np; i++) {
        if (pst[i] || ncols[i] == 0) continue;
        int want = b->workers > 0 && b->workers < ncols[i] ? b->workers : ncols[i];
        if (b->block && b->workers == 0) want = 1;
        auto &v = b->slots[i];
        while ((int)v.size() < want) {
            BatchSlot s;
            int st = make_slot(b->probs[i], true, s);
            if (st) break; // fewer slots: the columns are shared among those made
            v.push_back(s);
        }
        int ns = want < (int)v.size() ? want : (int)v.size();
        for (int k = 0; k < ns; k++) work.push_back({i, k, ns});
    }
    std::vector<amgh_solve_info> acc(work.size());
    std::vector<int> wst(work.size(), AMGH_OK);
    run_all(b, (int)work.size(), [&](int wi) {
        const Work &w = work[wi];
        amgh_problem *p = b->slots[w.prob][w.slot].h;
        amgh_solve_info &a = acc[wi];
        memset(&a, 0, sizeof(a));
        // block mode: one contiguous share of the columns per slot, one call
        int nc = ncols[w.prob], share = (nc + w.nslot - 1) / w.nslot;
        int c_lo = b->block ? w.slot * share : w.slot;
        int c_hi = b->block ? (c_lo + share < nc ? c_lo + share : nc) : nc;
        int step = b->block ? share : w.nslot;
        for (int c = c_lo; c < c_hi; c += step) {
            amgh_solve_info one;
            memset(&one, 0, sizeof(one));
            int s;
            if (b->block) {
                s = amgh_solve_block(p, yd[w.prob] + (int64_t)c * p->nv, c_hi - c, u[w.prob] + (int64_t)c * p->n,
                                     opts, &one);
            } else {
                s = amgh_set_yd(p, yd[w.prob] + (int64_t)c * p->nv, 1);
                if (s == AMGH_OK) s = amgh_solve(p, nullptr, u[w.prob] + (int64_t)c * p->n, nullptr, opts, &one);
            }
            a.outer_iters += one.outer_iters;
            a.hessian_applies += one.hessian_applies;
            a.inner_iters += one.inner_iters;
            a.mass_iters += one.mass_iters;
            a.refinements += one.refinements;
            a.coarse_iters += one.coarse_iters;
            a.fallbacks += one.fallbacks;
            a.t_solve_s += one.t_solve_s;
            a.final_relres = one.final_relres > a.final_relres ? one.final_relres : a.final_relres;
            a.hessian_levels = one.hessian_levels;
            if (s != AMGH_OK && wst[wi] == AMGH_OK) wst[wi] = s;
        }
    });
    // per problem: counters summed over its slots, status = its first error
    std::vector<amgh_solve_info> out(np);
    for (int i = 0; i < np; i++) {
        memset(&out[i], 0, sizeof(out[i]));
        out[i].status = pst[i];
        out[i].t_setup_s = b->probs[i]->t_setup;
    }
    for (size_t wi = 0; wi < work.size(); wi++) {
        amgh_solve_info &o = out[work[wi].prob];
        const amgh_solve_info &a = acc[wi];
        o.outer_iters += a.outer_iters;
        o.hessian_applies += a.hessian_applies;
        o.inner_iters += a.inner_iters;
        o.mass_iters += a.mass_iters;
        o.refinements += a.refinements;
        o.coarse_iters += a.coarse_iters;
        o.fallbacks += a.fallbacks;
        o.t_solve_s = a.t_solve_s > o.t_solve_s ? a.t_solve_s : o.t_solve_s;
        o.final_relres = a.final_relres > o.final_relres ? a.final_relres : o.final_relres;
        if (work[wi].slot == 0 || a.hessian_levels < o.hessian_levels) o.hessian_levels = a.hessian_levels;
        if (wst[wi] != AMGH_OK && o.status == AMGH_OK) o.status = wst[wi];
    }
    if (info)
        for (int i = 0; i < np; i++) info[i] = out[i];
    for (int i = 0; i < np; i++)
        if (out[i].status != AMGH_OK) return out[i].status;
    return AMGH_OK;
}

// The block width and slot count autotuner: every candidate -- one slot per
// desired state, or block solves of K = 8, 4 or 2 columns on 8/K slots per
// problem -- solves the whole batch once to capture its graphs and once more
// under the host clock; the fastest is kept for the batch's later solves.
extern "C" int amgh_batch_autotune(amgh_batch *b, const double *const *yd, const int *ncols, double *const *u,
                                   const amgh_solve_opts *opts, double *times, int *choice)
{
    if (!b) return AMGH_ERR_INVALID_ARG;
    static const int cand[4][2] = {{0, 0}, {1, 1}, {1, 2}, {1, 4}}; // {block, workers}
    int best = 0;
    double tbest = 0.0;
    for (int k = 0; k < 4; k++) {
        b->block = cand[k][0];
        b->workers = cand[k][1];
        TRY(amgh_batch_solve(b, yd, ncols, u, opts, nullptr));
        auto t0 = std::chrono::steady_clock::now();
        TRY(amgh_batch_solve(b, yd, ncols, u, opts, nullptr));
        double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (times) times[k] = t;
        if (k == 0 || t < tbest) {
            tbest = t;
            best = k;
        }
    }
    b->block = cand[best][0];
    b->workers = cand[best][1];
    if (choice) *choice = best;
    return AMGH_OK;
}

extern "C" void amgh_batch_destroy(amgh_batch *b)
{
    if (!b) return;
    for (size_t i = 0; i < b->slots.size(); i++) {
        auto &v = b->slots[i];
        for (size_t k = v.size(); k-- > 0;) {
            BatchSlot &s = v[k];
            if (!s.owned && s.h) {
                cudaStreamSynchronize(s.stream);
                amgh_set_stream(s.h, b->old_streams[i]);
                if (s.h->wait_ev) cudaEventDestroy(s.h->wait_ev);
                s.h->wait_ev = nullptr;
                s.h = nullptr;
            }
            slot_release(s);
        }
    }
    delete b;
}
