// serve.cpp -- placeholder for the serving loop (filled in with the batch path).
#include "../../include/eh.h"

#include <cstring>

extern void eh_set_error(const char *fmt, ...);

extern "C" {
eh_status eh_server_create(const eh_trie *, uint64_t, uint32_t, uint32_t, eh_server **out) {
    if (out) *out = nullptr;
    eh_set_error("serving is not available in this build");
    return EH_EINVAL;
}
eh_status eh_server_submit(eh_server *, eh_pattern, const uint32_t *, uint32_t, uint64_t *) { return EH_EINVAL; }
eh_status eh_server_poll(eh_server *, uint64_t, int *, uint64_t *, eh_status *) { return EH_EINVAL; }
eh_status eh_server_wait(eh_server *, uint64_t, uint32_t, uint64_t *, eh_status *) { return EH_EINVAL; }
eh_status eh_server_stats_get(eh_server *, eh_server_stats *) { return EH_EINVAL; }
void eh_server_destroy(eh_server *) {}
}
