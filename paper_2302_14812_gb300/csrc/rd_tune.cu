// Tuning cache of the deposit-shape autotuner (rd_autotune_shape): a JSON file that maps a problem
// key to the shape the tuner chose for it, so that later runs (and the batched form) take the shape
// without timing again.  Host code only.
//
// File layout:
//   {
//     "rd_shape_cache": 1,
//     "entries": {
//       "<key>": {"cells_per_cta": 256, "cells_per_thread": 2, "chunk": 4096, "group": 4, "ms": 147.8},
//       ...
//     }
//   }
// The key names the device (name and multiprocessor count) and the problem (cells, bins, particles,
// intervals, flags).  The file is read whole and rewritten whole through a temporary file and a
// rename, so a reader never sees a half-written file; two tuners writing one file at the same time
// may lose one of their entries.
#include <errno.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>

#include "rd_internal.cuh"

namespace rd {

namespace {

// Minimal JSON reader for the layout above: objects, strings, numbers, true/false/null; arrays
// are parsed and skipped.  Values of an entry other than numbers are ignored.
struct Reader {
    const char* p;
    const char* end;
    std::string err;

    void ws()
    {
        while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p;
    }
    bool lit(char c)
    {
        ws();
        if (p < end && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    bool fail(const char* what)
    {
        if (err.empty()) err = what;
        return false;
    }
    bool str(std::string& out)
    {
        ws();
        if (p >= end || *p != '"') return fail("expected a string");
        ++p;
        out.clear();
        while (p < end && *p != '"') {
            if (*p == '\\') {
                if (++p >= end) return fail("bad escape");
                const char c = *p;
                out.push_back(c == 'n' ? '\n' : c == 't' ? '\t' : c);
            } else {
                out.push_back(*p);
            }
            ++p;
        }
        if (p >= end) return fail("unterminated string");
        ++p;
        return true;
    }
    bool num(double& v)
    {
        ws();
        char* q = nullptr;
        v = strtod(p, &q);
        if (q == p || q > end) return fail("expected a number");
        p = q;
        return true;
    }
    // skip any value
    bool skip()
    {
        ws();
        if (p >= end) return fail("unexpected end");
        if (*p == '"') {
            std::string s;
            return str(s);
        }
        if (*p == '{' || *p == '[') {
            const char close = *p == '{' ? '}' : ']';
            const bool obj = *p == '{';
            ++p;
            if (lit(close)) return true;
            do {
                if (obj) {
                    std::string k;
                    if (!str(k) || !lit(':')) return fail("bad object");
                }
                if (!skip()) return false;
            } while (lit(','));
            return lit(close) ? true : fail("bad container");
        }
        for (const char* w : {"true", "false", "null"}) {
            const size_t n = strlen(w);
            if ((size_t)(end - p) >= n && strncmp(p, w, n) == 0) {
                p += n;
                return true;
            }
        }
        double v;
        return num(v);
    }
    bool entry(TuneEntry& e)
    {
        if (!lit('{')) return fail("expected an entry object");
        if (lit('}')) return true;
        do {
            std::string k;
            if (!str(k) || !lit(':')) return fail("bad entry");
            ws();
            if (p < end && (*p == '-' || (*p >= '0' && *p <= '9'))) {
                double v;
                if (!num(v)) return false;
                if (k == "cells_per_cta") e.cpc = (int)v;
                else if (k == "cells_per_thread") e.nc = (int)v;
                else if (k == "chunk") e.chunk = (int)v;
                else if (k == "group") e.group = (int)v;
                else if (k == "ms") e.ms = v;
            } else if (!skip()) {
                return false;
            }
        } while (lit(','));
        return lit('}') ? true : fail("bad entry end");
    }
    bool file(std::map<std::string, TuneEntry>& out)
    {
        if (!lit('{')) return fail("expected a JSON object");
        if (lit('}')) return true;
        do {
            std::string k;
            if (!str(k) || !lit(':')) return fail("bad top-level member");
            if (k == "entries") {
                if (!lit('{')) return fail("entries must be an object");
                if (!lit('}')) {
                    do {
                        std::string key;
                        TuneEntry e{};
                        if (!str(key) || !lit(':') || !entry(e)) return fail("bad entries");
                        out[key] = e;
                    } while (lit(','));
                    if (!lit('}')) return fail("bad entries end");
                }
            } else if (!skip()) {
                return false;
            }
        } while (lit(','));
        return lit('}') ? true : fail("bad end of file");
    }
};

std::string quote(const std::string& s)
{
    std::string o = "\"";
    for (char c : s) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o + "\"";
}

}  // namespace

bool tune_cache_load(const char* path, std::map<std::string, TuneEntry>& out, std::string& err)
{
    out.clear();
    FILE* f = fopen(path, "rb");
    if (!f) {
        if (errno == ENOENT) return true;            // no cache yet: empty
        err = std::string("cannot open ") + path + ": " + strerror(errno);
        return false;
    }
    std::string text;
    char buf[65536];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    fclose(f);
    Reader r{text.data(), text.data() + text.size(), {}};
    if (!r.file(out)) {
        err = std::string("malformed tuning cache ") + path + ": " + r.err;
        out.clear();
        return false;
    }
    return true;
}

bool tune_cache_store(const char* path, const std::string& key, const TuneEntry& e, std::string& err)
{
    std::map<std::string, TuneEntry> all;
    if (!tune_cache_load(path, all, err)) return false;
    all[key] = e;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) {
        err = std::string("cannot write ") + tmp + ": " + strerror(errno);
        return false;
    }
    fprintf(f, "{\n  \"rd_shape_cache\": 1,\n  \"entries\": {");
    bool first = true;
    for (const auto& kv : all) {
        fprintf(f, "%s\n    %s: {\"cells_per_cta\": %d, \"cells_per_thread\": %d, \"chunk\": %d, \"group\": %d, \"ms\": %.6g}",
                first ? "" : ",", quote(kv.first).c_str(), kv.second.cpc, kv.second.nc, kv.second.chunk,
                kv.second.group, kv.second.ms);
        first = false;
    }
    fprintf(f, "\n  }\n}\n");
    const bool ok = fflush(f) == 0;
    fclose(f);
    if (!ok || rename(tmp.c_str(), path) != 0) {
        err = std::string("cannot replace ") + path + ": " + strerror(errno);
        remove(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace rd
