// capi_internal.h -- helpers shared by the translation units of the C ABI.
#pragma once
#include <string>

namespace oocs {

// Record the text returned by oocs_last_error(NULL) for this host thread.
void set_last_error(const std::string &msg);

}  // namespace oocs
