// Thread-local error message behind ptycho_last_error().
#pragma once
#include <string>

int perr(int code, const std::string& msg);
