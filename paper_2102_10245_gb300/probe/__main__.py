"""Entry point of ``python -m paper_2102_10245_gb300.probe``."""
import sys

from . import main

sys.exit(main())
