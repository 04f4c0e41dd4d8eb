"""python -m roofline [--iters N]: one JSON line of measured issue rates."""
import argparse
import json

from . import measure

ap = argparse.ArgumentParser()
ap.add_argument("--iters", type=int, default=1024)
print(json.dumps(measure(ap.parse_args().iters)))
