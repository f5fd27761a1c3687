// capi_internal.h -- helpers shared by the translation units of the C ABI.
#pragma once
#include <string>

#include "../../include/oocs.h"

namespace oocs {

// Record the text returned by oocs_last_error(NULL) for this host thread.
void set_last_error(const std::string &msg);

// The status an entry point of the C ABI returns when an exception (a failed
// host allocation inside the library) reached it: OOCS_ERR_HOST_ALLOC, with
// the message recorded on ctx (or for oocs_last_error(NULL)) when possible.
// No exception leaves the C ABI.
oocs_status exception_status(oocs_ctx *ctx);

}  // namespace oocs
