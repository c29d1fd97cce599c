// Entry points declared in rbki.h whose implementation lives in later translation units.
// (placeholder: returns RBKI_E_UNSUPPORTED)
#include "plan.h"

using namespace rbki;

extern "C" {
rbki_status rbki_server_create(int32_t, size_t, int32_t, rbki_server**) {
    return set_error(RBKI_E_UNSUPPORTED, "server not built");
}
rbki_status rbki_submit(rbki_server*, const rbki_tensor*, const rbki_params*, const rbki_tucker_out*,
                        uint64_t*) {
    return set_error(RBKI_E_UNSUPPORTED, "server not built");
}
rbki_status rbki_poll(rbki_server*, uint64_t, rbki_status*, double*) {
    return set_error(RBKI_E_UNSUPPORTED, "server not built");
}
rbki_status rbki_cancel(rbki_server*, uint64_t) { return set_error(RBKI_E_UNSUPPORTED, "server not built"); }
rbki_status rbki_server_drain(rbki_server*, double) { return set_error(RBKI_E_UNSUPPORTED, "server not built"); }
rbki_status rbki_server_destroy(rbki_server*) { return set_error(RBKI_E_UNSUPPORTED, "server not built"); }
}
