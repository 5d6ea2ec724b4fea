// batch.cu -- native batch runtime: many independent control problems solved
// concurrently (one stream and one host worker thread per problem).
#include <string.h>

#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

struct amgh_batch {
    std::vector<amgh_problem *> probs;
    std::vector<cudaStream_t> streams;
    std::vector<void *> old_streams;
    int device = 0;
};

extern "C" int amgh_batch_create(amgh_problem *const *probs, int nprob, amgh_batch **out)
{
    if (!out || !probs || nprob <= 0) return AMGH_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < nprob; i++)
        if (!probs[i]) return AMGH_ERR_INVALID_ARG;
    amgh_batch *b = new (std::nothrow) amgh_batch();
    if (!b) return AMGH_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return AMGH_ERR_CUDA;
    }
    for (int i = 0; i < nprob; i++) {
        cudaStream_t s = 0;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            amgh_batch_destroy(b);
            return AMGH_ERR_CUDA;
        }
        b->probs.push_back(probs[i]);
        b->streams.push_back(s);
        b->old_streams.push_back((void *)probs[i]->stream);
        // work already queued on the old stream must finish before the new one runs
        cudaStreamSynchronize(probs[i]->stream);
        amgh_set_stream(probs[i], s);
    }
    *out = b;
    return AMGH_OK;
}

// run fn(i) for every problem on its own thread (device made current there)
template <typename F>
static void run_all(amgh_batch *b, F fn)
{
    std::vector<std::thread> th;
    th.reserve(b->probs.size());
    for (size_t i = 0; i < b->probs.size(); i++)
        th.emplace_back([b, i, &fn] {
            cudaSetDevice(b->device);
            fn((int)i);
        });
    for (auto &t : th) t.join();
}

extern "C" int amgh_batch_setup(amgh_batch *b, const amgh_amg_opts *amg)
{
    if (!b) return AMGH_ERR_INVALID_ARG;
    std::vector<int> st(b->probs.size(), AMGH_OK);
    run_all(b, [&](int i) {
        if (!b->probs[i]->setup_done) st[i] = amgh_amg_setup(b->probs[i], amg);
    });
    for (int s : st)
        if (s != AMGH_OK) return s;
    return AMGH_OK;
}

extern "C" int amgh_batch_solve(amgh_batch *b, const double *const *yd, const int *ncols, double *const *u,
                                const amgh_solve_opts *opts, amgh_solve_info *info)
{
    if (!b || !yd || !ncols || !u) return AMGH_ERR_INVALID_ARG;
    size_t np = b->probs.size();
    for (size_t i = 0; i < np; i++)
        if (ncols[i] < 0 || (ncols[i] > 0 && (!yd[i] || !u[i]))) return AMGH_ERR_INVALID_ARG;
    std::vector<int> st(np, AMGH_OK);
    std::vector<amgh_solve_info> acc(np);
    run_all(b, [&](int i) {
        amgh_problem *p = b->probs[i];
        amgh_solve_info &a = acc[i];
        memset(&a, 0, sizeof(a));
        if (!p->setup_done) {
            st[i] = amgh_amg_setup(p, nullptr);
            if (st[i]) return;
        }
        for (int c = 0; c < ncols[i]; c++) {
            int s = amgh_set_yd(p, yd[i] + (int64_t)c * p->nv, 1);
            amgh_solve_info one;
            memset(&one, 0, sizeof(one));
            if (s == AMGH_OK) s = amgh_solve(p, nullptr, u[i] + (int64_t)c * p->n, nullptr, opts, &one);
            a.outer_iters += one.outer_iters;
            a.hessian_applies += one.hessian_applies;
            a.inner_iters += one.inner_iters;
            a.mass_iters += one.mass_iters;
            a.refinements += one.refinements;
            a.t_solve_s += one.t_solve_s;
            a.final_relres = one.final_relres > a.final_relres ? one.final_relres : a.final_relres;
            a.t_setup_s = one.t_setup_s;
            if (s != AMGH_OK && st[i] == AMGH_OK) st[i] = s;
        }
        a.status = st[i];
    });
    if (info)
        for (size_t i = 0; i < np; i++) info[i] = acc[i];
    for (int s : st)
        if (s != AMGH_OK) return s;
    return AMGH_OK;
}

extern "C" void amgh_batch_destroy(amgh_batch *b)
{
    if (!b) return;
    for (size_t i = 0; i < b->probs.size(); i++) {
        cudaStreamSynchronize(b->streams[i]);
        amgh_set_stream(b->probs[i], b->old_streams[i]);
    }
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    delete b;
}
