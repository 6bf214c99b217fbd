// tune.cu -- the results of tile-shape tuning, shared by every context of
// the process and optionally kept in a text file: one line per result,
// "<key> <choice> <microseconds>", read when tuning is switched on with
// that file and appended to when a new key is tuned.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
}  // namespace

bool ibip_tune_get(const std::string &key, int *choice)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *choice = it->second;
    return true;
}

void ibip_tune_put(const std::string &key, int choice, double us, const char *path)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = choice;
    if (path && path[0]) {
        if (FILE *f = fopen(path, "a")) {
            fprintf(f, "%s %d %.3f\n", key.c_str(), choice, us);
            fclose(f);
        }
    }
}

int ibip_tune_load(const char *path)
{
    FILE *f = fopen(path, "r");
    if (!f) return 0;   // a missing file is an empty cache
    std::lock_guard<std::mutex> lk(g_tune_mu);
    char key[256];
    int choice = 0, n = 0;
    double us = 0.0;
    while (fscanf(f, "%255s %d %lf", key, &choice, &us) == 3) {
        g_tune[key] = choice;   // later lines win
        n++;
    }
    fclose(f);
    return n;
}
