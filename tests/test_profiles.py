"""The ncu summaries under profiles/ name commands that run committed files only:
every workload they profile is a case of bench.py --case, every ncu
command leaves the clocks alone (--clock-control none), and a full capture names
one kernel and a bounded launch count.  Checked as text; nothing runs."""
import pathlib
import re

ROOT = pathlib.Path(__file__).resolve().parent.parent
PROFILES = sorted((ROOT / "profiles").glob("*.md"))
BENCH_SRC = (ROOT / "bench.py").read_text()
CASES_SRC = BENCH_SRC[BENCH_SRC.index("def build_case("):BENCH_SRC.index("def run_case(")]


def _case_names():
    names = set(re.findall(r'name == "([a-z0-9-]+)"', CASES_SRC))
    for group in re.findall(r"name in \(([^)]*)\)", CASES_SRC):
        names.update(re.findall(r'"([a-z0-9-]+)"', group))
    return names


def test_there_are_profiles():
    assert len(PROFILES) >= 8


def test_profiled_workloads_are_committed_cases():
    known = _case_names()
    for p in PROFILES:
        text = p.read_text()
        assert "paper_2404_08867_gb300.cases" not in text, p.name
        for name in re.findall(r"bench\.py --case ([a-z0-9-]+)", text):
            assert name in known, (p.name, name)


def test_ncu_commands_leave_clocks_alone_and_are_bounded():
    for p in PROFILES:
        for line in p.read_text().splitlines():
            if not line.strip().startswith("ncu "):
                continue
            assert "--clock-control none" in line, (p.name, line)
            if "--set full" in line or "--section" in line:
                assert re.search(r"-k regex:\S+", line), (p.name, line)
                m = re.search(r"-c (\d+)", line)
                assert m and 1 <= int(m.group(1)) <= 3, (p.name, line)


def test_profiles_are_short_text():
    for p in PROFILES:
        assert p.stat().st_size < 16 * 1024, p.name
    assert not list((ROOT / "profiles").glob("*.ncu-rep"))
