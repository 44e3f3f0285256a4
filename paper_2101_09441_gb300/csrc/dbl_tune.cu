// Autotuner: picks the frontier schedule for this graph by measurement.
//
// Candidates are the team width (lanes that share one frontier task of up to
// kChunk edges: 4, 8, 16 or 32; or 1: one task per lane, the warp walking the
// concatenation of its tasks' edges) and whether frontier loops run as one
// persistent cooperative launch or level by level.  Each candidate runs the
// caller's sample insertion batch and query batch from the same snapshot
// (slot 3), timed with CUDA events on the stream; the index is restored after
// every trial, and the fastest candidate is kept in the index's options.
// Then, under that schedule, the label test's pairs per lane group
// (query_unroll 1, 2, 4) are timed on the query batch alone and the fastest
// is kept too.
#include <cstring>

#include "dbl_internal.cuh"

extern "C" dbl_status dbl_set_schedule(dbl_index *ix, int32_t team, int32_t persistent, int32_t query_unroll)
{
    if (!ix || (team != 1 && team != 4 && team != 8 && team != 16 && team != 32))
        return dbl::fail(ix, DBL_ERR_INVALID, "set_schedule: team must be 1, 4, 8, 16 or 32");
    if (query_unroll != 0 && query_unroll != 1 && query_unroll != 2 && query_unroll != 4)
        return dbl::fail(ix, DBL_ERR_INVALID, "set_schedule: query_unroll must be 0 (keep), 1, 2 or 4");
    ix->opt.team = team;
    if (query_unroll) ix->opt.query_unroll = query_unroll;
    ix->opt.flags = persistent ? (ix->opt.flags | DBL_FLAG_PERSISTENT) : (ix->opt.flags & ~DBL_FLAG_PERSISTENT);
    return DBL_OK;
}

extern "C" dbl_status dbl_autotune(dbl_index *ix, const int32_t *src, const int32_t *dst, int64_t b, const int32_t *u,
                                   const int32_t *v, int64_t q, uint8_t *ans, int32_t trials, double *report,
                                   void *stream)
{
    if (!ix || b < 0 || q < 0 || (b > 0 && (!src || !dst)) || (q > 0 && (!u || !v || !ans)) || trials < 1)
        return dbl::fail(ix, DBL_ERR_INVALID, "autotune: bad arguments");
    if (ix->poisoned) return dbl::fail(ix, DBL_ERR_POISONED, "autotune: index poisoned");
    cudaStream_t s = (cudaStream_t)stream;
    dbl_status st = dbl_snapshot(ix, 3, stream);
    if (st) return st;
    constexpr int kTeams = 5;
    const int teams[kTeams] = {1, 4, 8, 16, 32};
    const int32_t flags0 = ix->opt.flags, team0 = ix->opt.team;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int best_team = team0, best_persistent = (flags0 & DBL_FLAG_PERSISTENT) ? 1 : 0;
    int best_unroll = ix->opt.query_unroll;
    for (int p = 0; p < 2 && !st; ++p) {
        for (int t = 0; t < kTeams && !st; ++t) {
            ix->opt.team = teams[t];
            ix->opt.flags = (flags0 & ~(DBL_FLAG_PERSISTENT | DBL_FLAG_ASYNC | DBL_FLAG_TIMING)) |
                            (p ? DBL_FLAG_PERSISTENT : 0);
            float fastest = 3.4e38f;
            for (int r = 0; r < trials + 1 && !st; ++r) {  // first run warms up
                if ((st = dbl_restore(ix, 3, stream))) break;
                cudaEventRecord(e0, s);
                if (b && (st = dbl_insert_edges(ix, src, dst, b, stream))) break;
                if (q && (st = dbl_query(ix, u, v, q, ans, nullptr, stream))) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r && ms < fastest) fastest = ms;
            }
            const double avg = fastest;  // the fastest trial: least disturbed by anything else on the GPU
            if (report) report[p * kTeams + t] = avg;
            if (!st && avg < best) {
                best = avg;
                best_team = teams[t];
                best_persistent = p;
            }
        }
    }
    // label-test pairs per lane group, under the chosen schedule, on the query
    // batch alone (queries leave the index as it is)
    const int unrolls[3] = {1, 2, 4};
    if (q && !st) {
        ix->opt.team = best_team;
        ix->opt.flags = (flags0 & ~(DBL_FLAG_PERSISTENT | DBL_FLAG_ASYNC | DBL_FLAG_TIMING)) |
                        (best_persistent ? DBL_FLAG_PERSISTENT : 0);
        if (!(st = dbl_restore(ix, 3, stream)) && b) st = dbl_insert_edges(ix, src, dst, b, stream);
        double bq = 1e300;
        for (int i = 0; i < 3 && !st; ++i) {
            ix->opt.query_unroll = unrolls[i];
            float fastest = 3.4e38f;
            for (int r = 0; r < trials + 1 && !st; ++r) {
                cudaEventRecord(e0, s);
                if ((st = dbl_query(ix, u, v, q, ans, nullptr, stream))) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r && ms < fastest) fastest = ms;
            }
            if (report) report[13 + i] = fastest;
            if (!st && fastest < bq) {
                bq = fastest;
                best_unroll = unrolls[i];
            }
        }
    }
    ix->opt.query_unroll = best_unroll;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ix->opt.flags = (flags0 & ~DBL_FLAG_PERSISTENT) | (best_persistent ? DBL_FLAG_PERSISTENT : 0);
    ix->opt.team = best_team;
    dbl_status rs = dbl_restore(ix, 3, stream);
    if (st) return st;
    if (rs) return rs;
    if (report) {
        report[10] = best_team;
        report[11] = best_persistent;
        report[12] = best;
    }
    return dbl::read_status(ix, s);
}
