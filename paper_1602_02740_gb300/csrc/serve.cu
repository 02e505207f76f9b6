// Serving loop (see include/tc.h).  Placeholder entry points until the
// request loop lands: every call reports TC_EINVAL.
#include "../../include/tc.h"
#include "tc_ctx.h"

extern "C" tc_status tc_serve_submit(tc_ctx*, const uint32_t*, size_t, const uint32_t*, size_t,
                                     uint32_t*, uint64_t*) { return TC_EINVAL; }
extern "C" tc_status tc_serve_poll(tc_ctx*, uint64_t) { return TC_EINVAL; }
extern "C" tc_status tc_serve_stats(tc_ctx*, double*, double*, double*, uint64_t*) { return TC_EINVAL; }
extern "C" tc_status tc_serve_stop(tc_ctx*) { return TC_OK; }
