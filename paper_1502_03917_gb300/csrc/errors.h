// errors.h -- the library's error reporting, shared by its translation units
// (internal): records the message that mg_last_error() returns and passes the
// code through.
#pragma once
#include <string>

namespace aaomg {
int set_error(int code, const std::string& msg);
}  // namespace aaomg
