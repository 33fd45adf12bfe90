"""``python -m paper_2412_04514_gb300 points.npy -o cells.npz``: the command-line front-end."""
import sys

from .cli import main

sys.exit(main())
