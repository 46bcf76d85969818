// Partition-tree plans of the k-input multiplier (Section V-C).
#pragma once
#include <string>
#include <vector>

namespace ckks {

struct PlanNode {
    int size = 0;                 // inputs below this node
    std::vector<int> children;    // >= 0: node index; < 0: leaf -1 - input index
    int mu = 0;                   // m - 1 rescales
    bool root = false;
};

struct Plan {
    int k = 0;
    std::string text;
    std::vector<PlanNode> nodes;  // post-order, root last
    int depth = 0;
    int rs_units = 0;
};

const char *table_ii_partition(int k);
// 0 ok, -1 parse error, -2 depth rule broken
int plan_build(Plan &P, int k, const char *partition);
void plan_levels(const Plan &P, int level, std::vector<int> &lvl_in, std::vector<int> &lvl_out,
                 std::vector<int> &polys);

enum { kCostRsUnits = 0, kCostTransforms = 1, kCostPrecision = 2 };
// cost of a plan: Table II rescale units, or limb (I)NTTs at an input level
double plan_cost(const Plan &P, int criterion, int level, int K, int alpha);
// cheapest valid partition of k inputs; 0 ok, -1 none, -2 level too low
int plan_optimize(int k, int criterion, int level, int K, int alpha, std::string &best_text, double &best_cost);

}  // namespace ckks

// The plan handle of the C ABI.
struct ckks_plan {
    ckks::Plan p;
};
