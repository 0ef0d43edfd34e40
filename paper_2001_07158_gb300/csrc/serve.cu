// serve.cu -- batched decisions and the request server.
#include <vector>

#include "internal.h"

using namespace tmo;

struct tmotif_server {
    size_t budget = 0;
};

extern "C" {

int tmotif_decide_batch(const tmotif_graph_t *graphs, const tmotif_query *queries, uint32_t count,
                        tmotif_decision *out)
{
    if (count && (!graphs || !queries || !out)) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    for (uint32_t i = 0; i < count; i++) {
        int rc = tmotif_decide(graphs[i], &queries[i], &out[i]);
        if (rc != TMOTIF_OK) return rc;
    }
    return TMOTIF_OK;
}

int tmotif_server_create(size_t hbm_budget_bytes, tmotif_server_t *out)
{
    (void)hbm_budget_bytes;
    if (out) *out = nullptr;
    return fail(TMOTIF_ERR_UNSUPPORTED, "server not built yet").code;
}

int tmotif_submit(tmotif_server_t s, tmotif_graph_t g, const tmotif_query *q, int is_extract, uint64_t *ticket)
{
    (void)s; (void)g; (void)q; (void)is_extract; (void)ticket;
    return fail(TMOTIF_ERR_UNSUPPORTED, "server not built yet").code;
}

int tmotif_poll(tmotif_server_t s, uint64_t ticket, tmotif_decision *out, uint32_t *verts, uint32_t *times,
                int *done)
{
    (void)s; (void)ticket; (void)out; (void)verts; (void)times; (void)done;
    return fail(TMOTIF_ERR_UNSUPPORTED, "server not built yet").code;
}

void tmotif_server_destroy(tmotif_server_t s) { delete s; }

}  // extern "C"
