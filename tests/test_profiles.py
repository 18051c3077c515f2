"""The committed profile summaries (profiles/*.md, *.txt) are text that names
the commands which made them.  Those commands must stay safe to re-run:

* every ncu command leaves the GPU clocks alone (--clock-control none);
* every bench.py command a capture runs times one workload only
  (--headline-only, or the pass-based search's --method fm, which has no
  sub-records): otherwise bench.py also times every other workload, and ncu
  would serialise and profile each of their thousands of launches.

Commands are the indented or fenced code lines of the summaries, with
backslash continuations joined; shell variables (CMD="...") are expanded.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(path):
    lines, fenced = [], False
    for raw in open(path, encoding="utf-8").read().splitlines():
        if raw.strip().startswith("```"):
            fenced = not fenced
            continue
        if fenced or raw.startswith("    ") or raw.startswith("\t") or raw.startswith("  "):
            lines.append(raw.strip())
    cmds, cur = [], ""
    for ln in lines:
        cur = (cur + " " + ln) if cur else ln
        if cur.endswith("\\"):
            cur = cur[:-1].rstrip()
            continue
        cmds.append(cur)
        cur = ""
    if cur:
        cmds.append(cur)
    env = {}
    out = []
    for c in cmds:
        m = re.match(r'^([A-Z][A-Z0-9_]*)="(.*)"$', c)
        if m:
            env[m.group(1)] = m.group(2)
            continue
        for k, v in env.items():
            c = c.replace("$" + k, v)
        out.append(c)
    return out


def _summaries():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")))
    assert files
    return files


def test_every_ncu_command_leaves_clocks_alone():
    seen = 0
    for p in _summaries():
        for c in _commands(p):
            if re.search(r"(^|\s)ncu\s", c):
                seen += 1
                assert "--clock-control none" in c, f"{os.path.basename(p)}: {c}"
    assert seen > 0


def test_every_profiled_bench_command_times_one_workload():
    seen = 0
    for p in _summaries():
        for c in _commands(p):
            if re.search(r"(^|\s)(ncu\s.*)?python bench\.py", c) and "python bench.py" in c:
                seen += 1
                assert "--headline-only" in c or "--method fm" in c, f"{os.path.basename(p)}: {c}"
    assert seen > 0
