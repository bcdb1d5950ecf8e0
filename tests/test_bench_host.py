"""Host logic of bench.py that decides whether recorded ncu counters still
describe the stepper: the sources are compared without comments, so a comment
edit keeps the record and a code edit drops it."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strip_c_comments_keeps_code_and_literals():
    b = _bench()
    src = ('int a = 1; // trailing\n'
           '/* block\n   comment */ const char* u = "http://x /* not a comment */";\n'
           "\n"
           "char q = '\"'; float d = a / 2; // z\n"
           'asm("min.f32 %0, %1, %2, %3;" : "=f"(d));\n')
    out = b.strip_c_comments(src)
    assert "trailing" not in out and "block" not in out and "// z" not in out
    assert '"http://x /* not a comment */"' in out
    assert "char q = '\"'; float d = a / 2;" in out
    assert 'asm("min.f32 %0, %1, %2, %3;" : "=f"(d));' in out
    assert "\n\n" not in out


def test_comment_edit_keeps_hash_code_edit_changes_it():
    b = _bench()
    code = "__device__ float f(float x) {\n    return x * 2.0f;  // double it\n}\n"
    recomment = "// a new header comment\n__device__ float f(float x) {\n    return x * 2.0f;  /* twice */\n}\n"
    changed = "__device__ float f(float x) {\n    return x * 3.0f;  // double it\n}\n"
    assert b.strip_c_comments(code) == b.strip_c_comments(recomment)
    assert b.strip_c_comments(code) != b.strip_c_comments(changed)


def test_recorded_counters_match_current_sources():
    """profiles/stepper_counters.json and stepper_f64_counters.json carry the
    hash of the sources they were captured from; the committed tree must
    still match them (else the bench would silently drop the counters)."""
    b = _bench()
    assert b.stepper_counters("f32_kahan", 512, 64) is not None
    assert b.stepper_counters("f64", 256, 4, name="stepper_f64_counters.json") is not None
