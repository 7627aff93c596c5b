#include "errors.h"

#include "ptycho.h"

namespace {
thread_local std::string g_last_error;
}

int perr(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

extern "C" const char* ptycho_last_error(void) { return g_last_error.c_str(); }
