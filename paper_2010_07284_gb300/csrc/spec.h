// Specification text front end (host only): the command language of the
// paper's tool (Sec. 3) read into a node array for the formula compiler.
#pragma once
#include <string>
#include <vector>

#include "../../include/vl.h"

namespace vl {

struct TextSpec {
  std::vector<vl_node> nodes;       // topological order, shared sub-expressions
  std::vector<int32_t> roots;       // one per `save`, in order
  std::vector<std::string> loads;   // image names, in `load` order (image index)
  std::vector<std::string> sources; // the strings of those loads (what they name)
  std::vector<std::string> saves;   // output names, in `save` order (root index)
};

// Parse `src`; on failure returns false with "line L, column C: what" in *err.
bool parse_spec(const char* src, TextSpec* out, std::string* err);

}  // namespace vl
